"""Host check of the lane-product scheme of the lane-group kernels (csrc/dgx_stage3z.cuh, `xmatvec` and
`xcoef`), emulated lane by lane in numpy: a Q x Q product across the Q lanes of a group that differ in
one index bit field (stride 1 or Q) by recursive doubling -- one exchange with the partner i ^ 1, a
partial sum formed for the second partner i ^ 2 from the two values held, and its exchange -- must equal
the plain matrix-vector product for Q = 2 and 4, both strides, the matrix and its transpose.  This is
the identity the kernels rely on; the GPU parity tests check the kernels themselves."""
import numpy as np
import pytest


def _coef(M, i, Q):
    """the lane's coefficients: M[i][i], M[i][i^1] and, at Q = 4, M[i^2][i], M[i^2][i^1]"""
    c = [M[i, i], M[i, i ^ 1]]
    if Q == 4:
        c += [M[i ^ 2, i], M[i ^ 2, i ^ 1]]
    return c


def _lane_product(v, M, Q, stride):
    """32 lanes, groups of Q*Q lanes; lane index bit field selected by stride (1: low, Q: high)"""
    idx = lambda lane: (lane // stride) % Q
    coef = [_coef(M, idx(lane), Q) for lane in range(32)]
    w = np.array([v[lane ^ stride] for lane in range(32)])  # first exchange
    if Q == 2:
        return np.array([coef[l][0] * v[l] + coef[l][1] * w[l] for l in range(32)])
    part = np.array([coef[l][2] * v[l] + coef[l][3] * w[l] for l in range(32)])  # for partner i ^ 2
    recv = np.array([part[l ^ (2 * stride)] for l in range(32)])  # second exchange
    return np.array([coef[l][0] * v[l] + coef[l][1] * w[l] + recv[l] for l in range(32)])


@pytest.mark.parametrize("Q", [2, 4])
@pytest.mark.parametrize("transpose", [False, True])
def test_recursive_doubling_equals_matvec(Q, transpose):
    rng = np.random.default_rng(3 + Q)
    M = rng.standard_normal((Q, Q))
    Me = M.T if transpose else M
    for stride in (1, Q):
        v = rng.standard_normal(32)
        out = _lane_product(v, Me, Q, stride)
        for lane in range(32):
            i = (lane // stride) % Q
            base = lane - i * stride
            ref = sum(Me[i, j] * v[base + j * stride] for j in range(Q))
            assert abs(out[lane] - ref) < 1e-13


def test_a_wrong_partner_coefficient_fails():
    """planted: the partial sum formed with the lane's own row instead of its partner's"""
    Q = 4
    rng = np.random.default_rng(5)
    M = rng.standard_normal((Q, Q))
    v = rng.standard_normal(32)
    w = np.array([v[l ^ 1] for l in range(32)])
    part = np.array([M[l % Q, l % Q] * v[l] + M[l % Q, (l % Q) ^ 1] * w[l] for l in range(32)])
    recv = np.array([part[l ^ 2] for l in range(32)])
    out = np.array([M[l % Q, l % Q] * v[l] + M[l % Q, (l % Q) ^ 1] * w[l] + recv[l] for l in range(32)])
    ref = np.array([sum(M[l % Q, j] * v[l - l % Q + j] for j in range(Q)) for l in range(32)])
    assert np.abs(out - ref).max() > 1e-3
