"""SubApSnap online stage on GB300 (sm_103a): C-ABI library + thin binding.

``api`` mirrors the C entry points of include/subapsnap.h one to one;
``solver`` keeps the device copies of a problem's inputs alive next to a
context.  All arithmetic of the online stage runs in libsubapsnap.so.
"""
from . import api  # noqa: F401
