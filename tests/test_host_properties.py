"""Property tests of the library's host-side routines against the oracle (no GPU):
random inputs drawn by hypothesis, bit-identical answers required."""
import numpy as np
import pytest

try:  # an image without hypothesis skips these tests when they run, not at collection
    from hypothesis import given, settings, strategies as st
except ImportError:  # pragma: no cover
    given = None

from oracle import leverage, selection  # noqa: E402


def _api():
    from paper_2510_04825_gb300 import api
    try:
        api.lib()
    except Exception as e:  # pragma: no cover - the library is built by the test session
        pytest.skip(f"library not built: {e}")
    return api


if given is not None:
    @settings(max_examples=60, deadline=None)
    @given(n=st.integers(1, 300), s=st.integers(1, 200), seed=st.integers(0, 2 ** 31 - 1),
           power=st.sampled_from([1.0, 3.0, 8.0]))
    def test_leverage_sampler_matches_oracle(n, s, seed, power):
        api = _api()
        rng = np.random.default_rng(seed)
        scores = rng.uniform(0.0, 1.0, n) ** power
        scores[rng.integers(0, n)] += 1e-3  # never all zero
        u = rng.uniform(size=s)
        J, w = api.subapsnap_sample_rows_leverage(scores, s, u)
        Jo, wo = leverage.sample_rows(scores, s, u)
        np.testing.assert_array_equal(J, Jo)
        np.testing.assert_array_equal(w, wo)
        assert len(np.unique(J)) == len(J)


    @settings(max_examples=60, deadline=None)
    @given(m=st.integers(0, 200), dp=st.integers(1, 5), t=st.integers(1, 9), seed=st.integers(0, 2 ** 31 - 1),
           grid=st.booleans())
    def test_nearest_points_matches_oracle(m, dp, t, seed, grid):
        api = _api()
        rng = np.random.default_rng(seed)
        if grid:  # coarse lattices make exact ties common
            pts = rng.integers(0, 3, (t, dp)).astype(float)
            P = rng.integers(0, 3, (m, dp)).astype(float) / 2.0
        else:
            pts = rng.standard_normal((t, dp))
            P = rng.standard_normal((m, dp))
        np.testing.assert_array_equal(api.subapsnap_nearest_points(P.reshape(m, dp), pts),
                                      selection.nearest_points(P.reshape(m, dp), pts))


if given is None:  # pragma: no cover
    def test_leverage_sampler_matches_oracle():
        pytest.skip("hypothesis is not installed")

    def test_nearest_points_matches_oracle():
        pytest.skip("hypothesis is not installed")
