"""libnbody: GB300-native all-pairs N-body (arXiv 2203.08263's case study).

The compute path is the C-ABI shared library built from ``csrc/`` (see
``include/nbody.h``); :mod:`.nbody` is its thin Python binding and
:mod:`.autograd` the trajectory ``torch.autograd.Function``. Importing the
package itself loads nothing; the binding loads ``libnbody.so`` on first use
and raises if it is missing.
"""
__all__ = ["ics"]
