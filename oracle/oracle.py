"""ctypes wrapper of the CPU oracle (test infrastructure only).

Every function here forwards to oracle/cse_oracle.c; no arithmetic of the
method is done in Python.  Designs and tile sets are the plain containers of
paper_2212_10042_gb300.workloads (seeded input generators, no method maths).
"""
import ctypes as C
import functools

import numpy as np

from . import build as _build

STAT_IDS = {"one_arm_z": 0, "two_arm_pooled_z": 1, "bayes4": 2, "berry4": 3}
FAMILY_BINOMIAL = 0
FAMILY_NORMAL = 1


class _Design(C.Structure):
    _fields_ = [("stat", C.c_int32), ("d", C.c_int32), ("n_looks", C.c_int32),
                ("look_n", C.c_int32 * 3), ("p0", C.c_double), ("drop", C.c_double),
                ("seed", C.c_uint64), ("tnull", C.c_double * 4)]


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


@functools.lru_cache(maxsize=1)
def lib():
    L = C.CDLL(_build.build())
    u32p, i32p, i64p, dp = (C.POINTER(C.c_uint32), C.POINTER(C.c_int32),
                            C.POINTER(C.c_int64), C.POINTER(C.c_double))
    L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.orc_uniform.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]
    L.orc_uniform.restype = C.c_uint32
    L.orc_threshold.argtypes = [C.c_double]
    L.orc_threshold.restype = C.c_uint32
    L.orc_stat_one_arm.argtypes = [C.c_int32, C.c_int32, C.c_double]
    L.orc_stat_one_arm.restype = C.c_double
    L.orc_stat_two_arm.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32]
    L.orc_stat_two_arm.restype = C.c_double
    L.orc_bayes4_posterior.argtypes = [i32p, i32p, dp]
    L.orc_bayes4_stat.argtypes = [C.POINTER(_Design), i32p, C.c_uint32]
    L.orc_bayes4_stat.restype = C.c_double
    L.orc_counts.argtypes = [C.POINTER(_Design), u32p, C.c_uint32, i32p]
    L.orc_simulate.argtypes = [C.POINTER(_Design), C.c_int64, dp, u32p, i32p, C.c_double,
                               i64p, i64p, dp, dp, i64p]
    L.orc_simulate.restype = C.c_int
    L.orc_cp_upper.argtypes = [C.c_int64, C.c_int64, C.c_double]
    L.orc_cp_upper.restype = C.c_double
    L.orc_tilt_bound.argtypes = [C.c_int, C.c_int, dp, dp, dp, C.c_double, dp, dp]
    L.orc_tilt_bound_log.argtypes = [C.c_int, C.c_int, dp, dp, dp, C.c_double, dp, dp]
    L.orc_tilt_lower.argtypes = [C.c_int, C.c_int, dp, dp, dp, C.c_double, dp, dp]
    L.orc_cp_lower.argtypes = [C.c_int64, C.c_int64, C.c_double]
    L.orc_cp_lower.restype = C.c_double
    L.orc_alpha_prime.argtypes = [C.c_int, C.c_int, dp, dp, dp, C.c_double, dp, dp]
    L.orc_log_partition.argtypes = [C.c_int, C.c_int, dp, dp]
    L.orc_log_partition.restype = C.c_double
    L.orc_validate_bounds.argtypes = [C.POINTER(_Design), C.c_int64, dp, dp, i32p, i64p,
                                      C.c_double, dp, dp, dp]
    L.orc_validate_lower.argtypes = [C.POINTER(_Design), C.c_int64, dp, dp, i32p, i64p,
                                     C.c_double, dp, dp, dp]
    L.orc_berry_posterior.argtypes = [i32p, C.c_int32, dp, dp]
    L.orc_berry_stat.argtypes = [C.POINTER(_Design), i32p, C.c_uint32]
    L.orc_berry_stat.restype = C.c_double
    L.orc_tiebreak.argtypes = [C.c_uint64, C.c_uint32]
    L.orc_tiebreak.restype = C.c_uint32
    L.orc_simulate_rand.argtypes = [C.POINTER(_Design), C.c_int64, dp, u32p, i32p, C.c_double, C.c_uint32,
                                    i64p, i64p, dp]
    L.orc_simulate_rand.restype = C.c_int
    L.orc_calibrate_rand.argtypes = [C.POINTER(_Design), C.c_int64, dp, dp, u32p, i32p, C.c_double,
                                     dp, i64p, dp, u32p, u32p]
    L.orc_calibrate_rand.restype = C.c_double
    L.orc_calibrate.argtypes = [C.POINTER(_Design), C.c_int64, dp, dp, u32p, i32p, C.c_double,
                                dp, i64p, dp]
    L.orc_calibrate.restype = C.c_double
    L.orc_score_backward.argtypes = [C.c_int64, C.c_int, dp, dp, i32p, dp]
    L.orc_num_threads.restype = C.c_int
    return L


def _design(design):
    D = _Design()
    D.stat = STAT_IDS[design.stat]
    D.d = design.d
    D.n_looks = len(design.looks)
    for i, n in enumerate(design.looks):
        D.look_n[i] = n
    D.p0 = design.p0
    D.drop = design.drop
    D.seed = design.seed
    for i, t in enumerate(design.arm_null):
        D.tnull[i] = t
    return D


def num_threads():
    return lib().orc_num_threads()


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def uniform(seed, k, a, j):
    return lib().orc_uniform(seed, k, a, j)


def threshold(theta):
    return lib().orc_threshold(float(theta))


def stat_one_arm(x, n, p0=0.5):
    return lib().orc_stat_one_arm(x, n, p0)


def stat_two_arm(x0, x1, n0, n1):
    return lib().orc_stat_two_arm(x0, x1, n0, n1)


def bayes4_posterior(x, n):
    xa = np.ascontiguousarray(x, dtype=np.int32)
    na = np.ascontiguousarray(n, dtype=np.int32)
    P = np.zeros(3)
    lib().orc_bayes4_posterior(_p(xa, C.c_int32), _p(na, C.c_int32), _p(P, C.c_double))
    return P


def bayes4_stat(design, xl, null_mask):
    D = _design(design)
    x = np.zeros((3, 4), dtype=np.int32)
    x[:len(xl)] = xl
    return lib().orc_bayes4_stat(C.byref(D), _p(x, C.c_int32), null_mask)


def counts(design, theta, k):
    """Cumulative success counts x[look][arm] of sim k at parameter theta."""
    D = _design(design)
    t = np.array([threshold(th) for th in np.atleast_1d(theta)] + [0] * (4 - design.d),
                 dtype=np.uint32)
    x = np.zeros(12, dtype=np.int32)
    lib().orc_counts(C.byref(D), _p(t, C.c_uint32), k, _p(x, C.c_int32))
    return x.reshape(3, 4)[:len(design.looks), :design.d]


def simulate(design, tiles, lam, want_S=False):
    """Returns dict(R, Xrej, score[, S]) for every tile of `tiles`."""
    D = _design(design)
    th = np.ascontiguousarray(tiles.centers, dtype=np.float64)
    nm = np.ascontiguousarray(tiles.null_mask, dtype=np.uint32)
    K = np.ascontiguousarray(tiles.K, dtype=np.int32)
    n = len(K)
    R = np.zeros(n, dtype=np.int64)
    X = np.zeros((n, design.d), dtype=np.int64)
    G = np.zeros((n, design.d), dtype=np.float64)
    S = off = None
    if want_S:
        off = np.zeros(n + 1, dtype=np.int64)
        off[1:] = np.cumsum(K)
        S = np.zeros(int(off[-1]), dtype=np.float64)
    lib().orc_simulate(C.byref(D), n, _p(th, C.c_double), _p(nm, C.c_uint32), _p(K, C.c_int32),
                       float(lam), _p(R, C.c_int64), _p(X, C.c_int64), _p(G, C.c_double),
                       _p(S, C.c_double) if want_S else None,
                       _p(off, C.c_int64) if want_S else None)
    out = dict(R=R, Xrej=X, score=G)
    if want_S:
        out["S"] = [S[off[i]:off[i + 1]] for i in range(n)]
    return out


def cp_upper(R, N, delta):
    return lib().orc_cp_upper(int(R), int(N), float(delta))


def cp_lower(R, N, delta):
    """l with P(Binom(N, l) >= R) = delta (lower Clopper-Pearson); 0 for R = 0."""
    return lib().orc_cp_lower(int(R), int(N), float(delta))


def _vec(x, d):
    a = np.zeros(4)
    a[:d] = np.atleast_1d(np.asarray(x, dtype=np.float64))
    return a


def tilt_bound(theta0, h, a, nvec, family=FAMILY_BINOMIAL):
    d = len(np.atleast_1d(theta0))
    b, q = C.c_double(), C.c_double()
    lib().orc_tilt_bound(family, d, _p(_vec(nvec, d), C.c_double), _p(_vec(theta0, d), C.c_double),
                         _p(_vec(h, d), C.c_double), float(a), C.byref(b), C.byref(q))
    return b.value, q.value


def tilt_bound_log(theta0, h, loga, nvec, family=FAMILY_BINOMIAL):
    """log of the tilewise optimised Tilt-Bound from log a, and q*."""
    d = len(np.atleast_1d(theta0))
    b, q = C.c_double(), C.c_double()
    lib().orc_tilt_bound_log(family, d, _p(_vec(nvec, d), C.c_double), _p(_vec(theta0, d), C.c_double),
                             _p(_vec(h, d), C.c_double), float(loga), C.byref(b), C.byref(q))
    return b.value, q.value


def tilt_lower(theta0, h, l, nvec, family=FAMILY_BINOMIAL):
    """Optimised lower Tilt-Bound over the box from a lower value l at its centre, and q*."""
    d = len(np.atleast_1d(theta0))
    b, q = C.c_double(), C.c_double()
    lib().orc_tilt_lower(family, d, _p(_vec(nvec, d), C.c_double), _p(_vec(theta0, d), C.c_double),
                         _p(_vec(h, d), C.c_double), float(l), C.byref(b), C.byref(q))
    return b.value, q.value


def alpha_prime(theta0, h, alpha, nvec, family=FAMILY_BINOMIAL):
    d = len(np.atleast_1d(theta0))
    ap, q = C.c_double(), C.c_double()
    lib().orc_alpha_prime(family, d, _p(_vec(nvec, d), C.c_double), _p(_vec(theta0, d), C.c_double),
                          _p(_vec(h, d), C.c_double), float(alpha), C.byref(ap), C.byref(q))
    return ap.value, q.value


def log_partition(theta, nvec, family=FAMILY_BINOMIAL):
    d = len(np.atleast_1d(theta))
    return lib().orc_log_partition(family, d, _p(_vec(nvec, d), C.c_double),
                                   _p(_vec(theta, d), C.c_double))


def validate_bounds(design, tiles, R, delta):
    D = _design(design)
    th = np.ascontiguousarray(tiles.centers, dtype=np.float64)
    hw = np.ascontiguousarray(tiles.halfwidth, dtype=np.float64)
    K = np.ascontiguousarray(tiles.K, dtype=np.int32)
    Ra = np.ascontiguousarray(R, dtype=np.int64)
    n = len(K)
    u0, bnd, qs = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().orc_validate_bounds(C.byref(D), n, _p(th, C.c_double), _p(hw, C.c_double),
                              _p(K, C.c_int32), _p(Ra, C.c_int64), float(delta),
                              _p(u0, C.c_double), _p(bnd, C.c_double), _p(qs, C.c_double))
    return dict(u0=u0, bound=bnd, qstar=qs)


def validate_lower(design, tiles, R, delta):
    """Lower CP l0 at each centre and the optimised lower Tilt-Bound over each box."""
    D = _design(design)
    th = np.ascontiguousarray(tiles.centers, dtype=np.float64)
    hw = np.ascontiguousarray(tiles.halfwidth, dtype=np.float64)
    K = np.ascontiguousarray(tiles.K, dtype=np.int32)
    Ra = np.ascontiguousarray(R, dtype=np.int64)
    n = len(K)
    l0, low, qs = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().orc_validate_lower(C.byref(D), n, _p(th, C.c_double), _p(hw, C.c_double),
                             _p(K, C.c_int32), _p(Ra, C.c_int64), float(delta),
                             _p(l0, C.c_double), _p(low, C.c_double), _p(qs, C.c_double))
    return dict(l0=l0, lower=low, qstar=qs)


def berry_posterior(x, n, tnull):
    """P(theta_i > 0 | x) for the four basket arms (offset log-odds)."""
    xa = np.ascontiguousarray(x, dtype=np.int32)
    ta = np.ascontiguousarray(tnull, dtype=np.float64)
    P = np.zeros(4)
    lib().orc_berry_posterior(_p(xa, C.c_int32), int(n), _p(ta, C.c_double), _p(P, C.c_double))
    return P


def berry_stat(design, x, null_mask):
    D = _design(design)
    xa = np.ascontiguousarray(x, dtype=np.int32)
    return lib().orc_berry_stat(C.byref(D), _p(xa, C.c_int32), int(null_mask))


def tiebreak(seed, k):
    """The tie-break word of sim k (randomised test)."""
    return int(lib().orc_tiebreak(int(seed), int(k)))


def simulate_rand(design, tiles, lam, c):
    """R, Xrej, score under the randomised rule: reject iff S < lam or (S == lam and w < c)."""
    D = _design(design)
    th = np.ascontiguousarray(tiles.centers, dtype=np.float64)
    nm = np.ascontiguousarray(tiles.null_mask, dtype=np.uint32)
    K = np.ascontiguousarray(tiles.K, dtype=np.int32)
    n = len(K)
    R = np.zeros(n, dtype=np.int64)
    X = np.zeros((n, design.d), dtype=np.int64)
    G = np.zeros((n, design.d), dtype=np.float64)
    lib().orc_simulate_rand(C.byref(D), n, _p(th, C.c_double), _p(nm, C.c_uint32), _p(K, C.c_int32),
                            float(lam), int(c), _p(R, C.c_int64), _p(X, C.c_int64), _p(G, C.c_double))
    return dict(R=R, Xrej=X, score=G)


def calibrate_rand(design, tiles, alpha):
    """Randomised calibration: per tile the k-th smallest (S, w) pair, and the lexicographic minimum."""
    D = _design(design)
    th = np.ascontiguousarray(tiles.centers, dtype=np.float64)
    hw = np.ascontiguousarray(tiles.halfwidth, dtype=np.float64)
    nm = np.ascontiguousarray(tiles.null_mask, dtype=np.uint32)
    K = np.ascontiguousarray(tiles.K, dtype=np.int32)
    n = len(K)
    ap, kk, lt = np.zeros(n), np.zeros(n, dtype=np.int64), np.zeros(n)
    ct = np.zeros(n, dtype=np.uint32)
    cs = C.c_uint32()
    lam = lib().orc_calibrate_rand(C.byref(D), n, _p(th, C.c_double), _p(hw, C.c_double),
                                   _p(nm, C.c_uint32), _p(K, C.c_int32), float(alpha),
                                   _p(ap, C.c_double), _p(kk, C.c_int64), _p(lt, C.c_double),
                                   _p(ct, C.c_uint32), C.byref(cs))
    return dict(alpha_prime=ap, k=kk, lambda_tile=lt, c_tile=ct, lam=lam, c=int(cs.value))


def calibrate(design, tiles, alpha):
    D = _design(design)
    th = np.ascontiguousarray(tiles.centers, dtype=np.float64)
    hw = np.ascontiguousarray(tiles.halfwidth, dtype=np.float64)
    nm = np.ascontiguousarray(tiles.null_mask, dtype=np.uint32)
    K = np.ascontiguousarray(tiles.K, dtype=np.int32)
    n = len(K)
    ap, kk, lt = np.zeros(n), np.zeros(n, dtype=np.int64), np.zeros(n)
    lam = lib().orc_calibrate(C.byref(D), n, _p(th, C.c_double), _p(hw, C.c_double),
                              _p(nm, C.c_uint32), _p(K, C.c_int32), float(alpha),
                              _p(ap, C.c_double), _p(kk, C.c_int64), _p(lt, C.c_double))
    return dict(alpha_prime=ap, k=kk, lambda_tile=lt, lam=lam)


def score_backward(grad_out, score, K):
    g = np.ascontiguousarray(grad_out, dtype=np.float64)
    s = np.ascontiguousarray(score, dtype=np.float64)
    Ka = np.ascontiguousarray(K, dtype=np.int32)
    n, d = s.shape
    out = np.zeros((n, d))
    lib().orc_score_backward(n, d, _p(g, C.c_double), _p(s, C.c_double), _p(Ka, C.c_int32),
                             _p(out, C.c_double))
    return out
