"""Tolerances shared by the GPU parity tests.

Modularity (Eq. 1) is accumulated in fp64 on both sides, in different orders, so the
CUDA path must agree with the oracle within 1e-9 relative.  Where the oracle's Q is
exactly 0 (one community: sigma_c / 2m and (Sigma_c / 2m)^2 are both exactly 1 for
integer-valued weights, whose fp64 sums are exact on both sides) a relative bound is
empty, and the CUDA path must give |Q| <= 1e-15 instead.
"""

Q_RTOL = 1e-9
Q_ATOL_AT_ZERO = 1e-15


def q_close(q: float, ref: float) -> bool:
    if ref == 0.0:
        return abs(q) <= Q_ATOL_AT_ZERO
    return abs(q - ref) <= Q_RTOL * abs(ref)
