"""The learned surrogate (not in the paper): kernels against the float64 oracle.

* Gradients of one forward/backward pass equal the oracle's (oracle/mlp.py, itself
  pinned by finite differences) evaluated with the same bfloat16-rounded weights:
  the device accumulates in float32, so the bound is 2e-3 relative per tensor
  (norm-wise), far above float32 rounding over a batch of 512 and far below
  any wrong index or transposed operand.
* Training on coefficient vectors from the online stage lowers the loss.
* The gate accepts exactly the predictions whose float64 subsampled residual,
  evaluated by the oracle, is <= tol (parameters within 1e-9 relative of the
  threshold are not compared); gate_tol = 0 reproduces the exact solve.
* The gain over the method without the network is measured and reported.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import mlp as omlp, online  # noqa: E402
from paper_2510_04825_gb300 import api  # noqa: E402
from paper_2510_04825_gb300.solver import AffineSolver  # noqa: E402

from _problems import Case  # noqa: E402


def bf16_round(a):
    """Round-to-nearest-even to bfloat16, returned as float64."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(theta, din, h, dout):
    shapes = [(h, din), (h,), (h, h), (h,), (dout, h), (dout,)]
    out, o = [], 0
    for sh in shapes:
        n = int(np.prod(sh))
        out.append(theta[o:o + n].reshape(sh).astype(np.float64))
        o += n
    return out


@pytest.fixture(scope="module")
def case():
    return Case("diffusion_2d", N=40, r=60, s=120, m=600)


@pytest.mark.parametrize("B,f32_out", [(512, 0), (1000, 0), (1000, 1), (64, 1)],
                         ids=["b512", "b1000-ragged", "b1000-f32-output-layer", "b64-f32-output-layer"])
def test_gradients_match_oracle(case, B, f32_out):
    """All products on the tensor cores (bfloat16 operands, float32 activations as two
    bfloat16 terms, float32 accumulation): one forward/backward against the oracle.  B
    covers one K block, a ragged batch split over many CTAs (split-K weight gradients),
    and the float32 output layer (SAS_OPT_SURROGATE_F32_OUT: the oracle then takes W3
    unrounded)."""
    p = case.prob
    solver = AffineSolver(p, case.S, case.J, mode=api.SAS_MODE_MIXED, device="cuda")
    api.subapsnap_set_option(solver.ctx, api.SAS_OPT_SURROGATE_F32_OUT, f32_out)
    nparam = api.subapsnap_surrogate_weights(solver.ctx, False)  # creates the network
    rng = np.random.default_rng(0)
    theta = np.zeros(nparam, dtype=np.float32)
    api.subapsnap_surrogate_weights(solver.ctx, True, theta)
    theta += (0.05 * rng.standard_normal(nparam)).astype(np.float32)  # non-trivial biases too
    api.subapsnap_surrogate_weights(solver.ctx, False, theta)
    X = rng.uniform(-1, 1, (B, p.dp))
    Yn = rng.standard_normal((B, p.r))
    loss, g = api.subapsnap_surrogate_grad(solver.ctx, torch.from_numpy(X).cuda(),
                                           torch.from_numpy(Yn).cuda(), nparam)
    W1, b1, W2, b2, W3, b3 = unpack(theta, p.dp, 256, p.r)
    params = [(bf16_round(W1), b1), (bf16_round(W2), b2), (W3 if f32_out else bf16_round(W3), b3)]
    # the device feeds float32 inputs: round them the same way
    Xf = X.astype(np.float32).astype(np.float64)
    Yf = Yn.astype(np.float32).astype(np.float64)
    loss_o, grads = omlp.loss_and_grads(params, Xf, Yf)
    assert abs(loss - loss_o) <= 1e-5 * loss_o
    gd = unpack(g, p.dp, 256, p.r)
    go = [grads[0][0], grads[0][1], grads[1][0], grads[1][1], grads[2][0], grads[2][1]]
    for k, (a, b) in enumerate(zip(gd, go)):
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        print(f"grad tensor {k}: rel err {rel:.2e}")
        assert rel <= 2e-3, (k, rel)
    solver.close()


def test_predictions_with_anchors_match_oracle(case):
    """Prediction = nearest anchor's y + network output (denormalised): the nearest anchor
    (input scaling, lowest index on ties) must equal numpy's choice exactly, and y_hat the
    oracle's float64 forward pass of the same weights within float32-class error."""
    p = case.prob
    solver = AffineSolver(p, case.S, case.J, mode=api.SAS_MODE_MIXED, device="cuda")
    rng = np.random.default_rng(4)
    na, ntrain = 37, 512
    Pa = rng.uniform(0.0, 1.0, (na, p.dp))
    Pa[5] = Pa[3]  # a duplicate anchor: the lower index wins
    Ya = rng.standard_normal((na, p.r))
    api.subapsnap_surrogate_set_anchors(solver.ctx, torch.from_numpy(Pa).cuda(), torch.from_numpy(Ya).cuda())
    Ptr = rng.uniform(0.0, 1.0, (ntrain, p.dp))
    Ytr = rng.standard_normal((ntrain, p.r))
    # zero epochs: fixes the normalisation (from the deviations) and the anchors only
    api.subapsnap_surrogate_train(solver.ctx, torch.from_numpy(Ptr).cuda(), torch.from_numpy(Ytr).cuda(),
                                  0, 256, 1e-3, seed=3)
    nparam = api.subapsnap_surrogate_weights(solver.ctx, False)
    theta = np.zeros(nparam, dtype=np.float32)
    norm = np.zeros(2 * (p.dp + p.r))
    api.subapsnap_surrogate_weights(solver.ctx, True, theta, norm)
    c, hw = norm[:p.dp], norm[p.dp:2 * p.dp]
    mu, sd = norm[2 * p.dp:2 * p.dp + p.r], norm[2 * p.dp + p.r:]
    # the normalisation was fitted to the deviations from the nearest anchors
    def nearest(P):
        d2 = (((P[:, None, :] - Pa[None, :, :]) / hw) ** 2).sum(axis=2)
        return d2.argmin(axis=1)
    dev = Ytr - Ya[nearest(Ptr)]
    np.testing.assert_allclose(mu, dev.mean(axis=0), rtol=1e-12, atol=1e-12)
    m = 300
    P = rng.uniform(0.0, 1.0, (m, p.dp))
    P[7] = Pa[3]
    Yhat = torch.empty((m, p.r), dtype=torch.float64, device="cuda")
    api.subapsnap_surrogate_predict(solver.ctx, torch.from_numpy(P).cuda(), m, Yhat)
    torch.cuda.synchronize()
    W1, b1, W2, b2, W3, b3 = unpack(theta, p.dp, 256, p.r)
    params = [(bf16_round(W1), b1), (bf16_round(W2), b2), (bf16_round(W3), b3)]
    Xn = ((P - c) / hw).astype(np.float32).astype(np.float64)
    out, _ = omlp.forward(params, Xn)
    nn = nearest(P)
    assert nn[7] == 3
    ref = Ya[nn] + mu + sd * out
    net = (Yhat.cpu().numpy() - Ya[nn] - mu) / sd
    rel = np.linalg.norm(net - out, axis=1) / np.linalg.norm(out, axis=1)
    print(f"anchored predictions: network output rel err max {rel.max():.2e}")
    assert rel.max() <= 1e-4
    np.testing.assert_allclose(Yhat.cpu().numpy(), ref, rtol=0, atol=1e-4 * np.abs(ref).max())
    solver.close()


def train(case, solver, ntrain=4096, epochs=60):
    p = case.prob
    rng = np.random.default_rng(5)
    Ptr = rng.uniform(0.0, 1.0, (ntrain, p.dp))
    Pd = torch.from_numpy(Ptr).cuda()
    Yd = torch.empty((ntrain, p.r), dtype=torch.float64, device="cuda")
    solver.solve(Pd, api.SAS_OUT_Y, Yd)  # training targets from the online stage itself
    losses = api.subapsnap_surrogate_train(solver.ctx, Pd, Yd, epochs, 256, 2e-3, seed=1)
    return losses


def test_training_and_gate(case):
    p = case.prob
    solver = AffineSolver(p, case.S, case.J, mode=api.SAS_MODE_MIXED, device="cuda")
    losses = train(case, solver)
    print(f"surrogate loss: first epoch {losses[0]:.3e}, last {losses[-1]:.3e}")
    assert losses[-1] < 0.05 * losses[0]
    params = p.test_params
    m = params.shape[0]
    P = torch.from_numpy(np.ascontiguousarray(params)).cuda()
    Yhat = torch.empty((m, p.r), dtype=torch.float64, device="cuda")
    api.subapsnap_surrogate_predict(solver.ctx, P, m, Yhat)
    torch.cuda.synchronize()
    Yh = Yhat.cpu().numpy()
    rho_hat = np.array([online.subsampled_residual(p, case.S, case.J, prm, y) for prm, y in zip(params, Yh)])
    tol = float(np.median(rho_hat))  # a threshold that splits the batch
    out = torch.empty((m, p.r), dtype=torch.float64, device="cuda")
    flags = torch.zeros(m, dtype=torch.int32, device="cuda")
    rho = torch.empty(m, dtype=torch.float64, device="cuda")
    acc = api.subapsnap_solve_batch_surrogate(solver.ctx, P, m, api.SAS_OUT_Y, out, flags, rho, tol)
    torch.cuda.synchronize()
    fl = flags.cpu().numpy()
    took = (fl & api.SAS_FLAG_SURROGATE) != 0
    clear = np.abs(rho_hat - tol) > 1e-9 * tol
    np.testing.assert_array_equal(took[clear], (rho_hat <= tol)[clear])
    assert acc == took.sum() and 0 < acc < m
    Y = out.cpu().numpy()
    np.testing.assert_array_equal(Y[took], Yh[took])  # accepted predictions pass through
    Yo, rho_o = case.oracle_solve(params[~took])
    err = np.linalg.norm(Y[~took] - Yo, axis=1) / np.linalg.norm(Yo, axis=1)
    assert err.max() <= 1e-8  # rejected ones are solved exactly (mixed form)
    # gate_tol = 0: everything falls back, identical to the exact solve
    Yex = torch.empty_like(out)
    solver.solve(P, api.SAS_OUT_Y, Yex)
    acc0 = api.subapsnap_solve_batch_surrogate(solver.ctx, P, m, api.SAS_OUT_Y, out, None, None, 0.0)
    torch.cuda.synchronize()
    assert acc0 == 0
    np.testing.assert_array_equal(out.cpu().numpy(), Yex.cpu().numpy())
    solver.close()


def test_surrogate_gain_is_measured(case):
    """What the network buys: acceptance rate and time against the exact solve, per threshold."""
    p = case.prob
    solver = AffineSolver(p, case.S, case.J, mode=api.SAS_MODE_MIXED, device="cuda")
    train(case, solver)
    rng = np.random.default_rng(9)
    m = 8192
    P = torch.from_numpy(rng.uniform(0, 1, (m, p.dp))).cuda()
    out = torch.empty((m, p.r), dtype=torch.float64, device="cuda")

    def timeit(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    t_exact = timeit(lambda: solver.solve(P, api.SAS_OUT_Y, out))
    rows = []
    for tol in (1e-6, 1e-5, 1e-4, 1e-3, 1e-2):
        acc = [0]

        def run():
            acc[0] = api.subapsnap_solve_batch_surrogate(solver.ctx, P, m, api.SAS_OUT_Y, out, None, None, tol)
        t = timeit(run)
        rows.append((tol, acc[0] / m, t_exact / t))
    for tol, rate, gain in rows:
        print(f"gate {tol:.0e}: accepted {100 * rate:5.1f}%  speed vs exact solve {gain:.2f}x")
    # the fully rejecting threshold costs one prediction and one residual more than the exact solve
    assert all(0.0 <= rate <= 1.0 for _, rate, _ in rows)
    solver.close()
