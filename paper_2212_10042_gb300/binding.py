"""Thin ctypes binding of libcse_gb300.so (include/cse.h), same names as the C ABI.

Argument marshalling only: tensors are passed as raw device pointers and every
step of the method runs in the library's CUDA kernels.  There is no fallback:
if the library cannot be loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import functools
import math
import os

import numpy as np
import torch

from . import build as _build
from . import workloads as W

STAT_IDS = {"one_arm_z": 0, "two_arm_pooled_z": 1, "bayes4": 2, "berry4": 3}
OPT_BAYES_DIRECT = 1
OPT_PLAIN = 2
OPT_SIM_THREADS = 3
OPT_CELLS_BOX = 4
OPT_PDL = 5
OPT_SIM_TILES = 7
STATUS = {0: "ok", -1: "invalid argument", -2: "unsupported design", -3: "device allocation failed",
          -4: "CUDA error", -5: "bounded device wait timed out", -6: "device-side argument check failed",
          -7: "request exceeds the fixed scratch capacity"}


class CseError(RuntimeError):
    def __init__(self, fn, status):
        super().__init__("%s failed: %s (%d)" % (fn, STATUS.get(status, "unknown"), status))
        self.status = status


class cse_design(C.Structure):
    _fields_ = [("stat", C.c_int32), ("d", C.c_int32), ("n_looks", C.c_int32),
                ("look_n", C.c_int32 * 3), ("p0", C.c_double), ("drop", C.c_double),
                ("arm_null", C.c_double * 4)]


class cse_tiles(C.Structure):
    _fields_ = [("n_tiles", C.c_int64), ("n_axis", C.c_int32 * 4), ("axis", C.c_void_p * 4),
                ("center_idx", C.c_void_p), ("halfwidth", C.c_void_p), ("null_mask", C.c_void_p),
                ("K", C.c_void_p), ("K_max", C.c_int32)]


_P = C.c_void_p


@functools.lru_cache(maxsize=1)
def lib() -> C.CDLL:
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libcse_gb300.so is not built (%s); run __graft_entry__.build()" % path)
    L = C.CDLL(path)
    L.cse_create.argtypes = [C.POINTER(_P), C.POINTER(cse_design), C.c_uint64, C.c_int32, _P]
    L.cse_destroy.argtypes = [_P]
    L.cse_simulate_tiles.argtypes = [_P, C.POINTER(cse_tiles), C.c_double, _P, _P, _P, _P]
    L.cse_validate.argtypes = [_P, C.POINTER(cse_tiles), C.c_double, C.c_double, _P, _P, _P, _P, _P, _P, _P]
    L.cse_validate_rand.argtypes = [_P, C.POINTER(cse_tiles), C.c_double, C.c_uint32, C.c_double, _P, _P, _P, _P,
                                    _P, _P, _P]
    L.cse_calibrate_rand.argtypes = [_P, C.POINTER(cse_tiles), C.c_double, _P, _P, _P, _P, _P, _P]
    L.cse_validate_lower.argtypes = [_P, C.POINTER(cse_tiles), C.c_double, C.c_double, _P, _P, _P, _P, _P, _P, _P]
    L.cse_validate_band.argtypes = [_P, C.POINTER(cse_tiles), C.c_double, C.c_double, _P, _P, _P, _P, _P, _P, _P,
                                    _P]
    L.cse_calibrate.argtypes = [_P, C.POINTER(cse_tiles), C.c_double, _P, _P, C.POINTER(C.c_double), _P]
    L.cse_step.argtypes = [_P, C.POINTER(cse_tiles), C.c_double, C.c_double, C.c_double] + [_P] * 10
    L.cse_score_backward.argtypes = [C.c_int64, C.c_int32, _P, _P, _P, _P, _P]
    L.cse_sync.argtypes = [_P, _P]
    L.cse_reseed.argtypes = [_P, C.c_uint64, _P]
    L.cse_statistics.argtypes = [_P, C.POINTER(cse_tiles), _P, _P, _P]
    L.cse_set_option.argtypes = [_P, C.c_int, C.c_int64]
    L.cse_autotune.argtypes = [_P, C.POINTER(cse_tiles), C.c_double, C.c_double, C.POINTER(C.c_int32),
                               C.POINTER(C.c_int32), _P]
    L.cse_profile_enable.argtypes = [_P, C.c_int]
    L.cse_profile_only.argtypes = [_P, C.c_char_p]
    L.cse_profile_read.argtypes = [_P, C.POINTER(C.c_char_p), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_double), C.c_int]
    L.cse_simulate_tiles_static.argtypes = [C.POINTER(cse_design), C.c_uint64, C.POINTER(cse_tiles), C.c_double,
                                            _P, _P, _P, _P]
    L.cse_type1_error.argtypes = [_P, C.c_int64, _P, _P, _P, C.c_int32, C.c_double, _P, _P, _P, _P, _P]
    L.cse_probe_peak.argtypes = [C.c_int, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), _P]
    L.cse_status_str.argtypes = [C.c_int]
    L.cse_status_str.restype = C.c_char_p
    L.cse_launch_count.argtypes = [_P]
    L.cse_launch_count.restype = C.c_int64
    return L


def _check(fn, st):
    if st != 0:
        raise CseError(fn, st)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def make_design(design: W.Design) -> cse_design:
    D = cse_design()
    D.stat = STAT_IDS[design.stat]
    D.d = design.d
    D.n_looks = len(design.looks)
    for i, n in enumerate(design.looks):
        D.look_n[i] = n
    D.p0 = design.p0
    D.drop = design.drop
    for a, t in enumerate(design.arm_null):
        D.arm_null[a] = t
    return D


def _per_point(v, n, np_dtype, torch_dtype, dev):
    """A per-point device array: a device tensor as given (same dtype width), or an
    int for every point, copied from the host (no device kernel)."""
    if isinstance(v, torch.Tensor):
        if v.numel() != n or v.element_size() != 4 or not v.is_contiguous() or v.device != dev:
            raise TypeError("per-point arrays must be contiguous 32-bit device tensors of length n")
        return v
    return torch.from_numpy(np.full(n, int(v), dtype=np_dtype).view(np.int32)).to(dev)


class DeviceTiles:
    """A tile set resident on the GPU (axis-indexed form of include/cse.h)."""

    def __init__(self, tiles: W.TileSet, device="cuda"):
        dev = torch.device(device)
        self.d = tiles.d
        self.n_tiles = tiles.n_tiles
        self.K_max = tiles.K_max
        self.axis = [torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
                     for a in tiles.axis]
        self.idx = torch.as_tensor(np.ascontiguousarray(tiles.idx), dtype=torch.int32, device=dev)
        self.halfwidth = torch.as_tensor(np.ascontiguousarray(tiles.halfwidth), dtype=torch.float64, device=dev)
        self.null_mask = torch.as_tensor(np.ascontiguousarray(tiles.null_mask).view(np.int32), device=dev)
        self.K = torch.as_tensor(np.ascontiguousarray(tiles.K), dtype=torch.int32, device=dev)
        self._struct = self._make_struct()

    @classmethod
    def from_tensors(cls, axis, idx, halfwidth, null_mask, K, K_max):
        self = cls.__new__(cls)
        self.d = idx.shape[1]
        self.n_tiles = idx.shape[0]
        self.K_max = int(K_max)
        self.axis, self.idx, self.halfwidth, self.null_mask, self.K = axis, idx, halfwidth, null_mask, K
        self._struct = self._make_struct()
        return self

    def _make_struct(self):
        T = cse_tiles()
        T.n_tiles = self.n_tiles
        for a in range(self.d):
            T.n_axis[a] = self.axis[a].numel()
            T.axis[a] = self.axis[a].data_ptr()
        T.center_idx = self.idx.data_ptr()
        T.halfwidth = self.halfwidth.data_ptr()
        T.null_mask = self.null_mask.data_ptr()
        T.K = self.K.data_ptr()
        T.K_max = self.K_max
        return T

    @property
    def struct(self):
        return self._struct

    def centers(self):
        return torch.stack([self.axis[a][self.idx[:, a].long()] for a in range(self.d)], dim=1)


class Context:
    """cse_create / cse_destroy around one design, seed and K_max."""

    def __init__(self, design: W.Design, seed: int = None, K_max: int = 1 << 16, stream=None):
        self.design = design
        self.seed = design.seed if seed is None else seed
        self.K_max = int(K_max)
        self._h = C.c_void_p()
        D = make_design(design)
        _check("cse_create", lib().cse_create(C.byref(self._h), C.byref(D), self.seed, self.K_max,
                                              _stream(stream)))

    def close(self):
        if self._h:
            lib().cse_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def launch_count(self) -> int:
        return lib().cse_launch_count(self._h)

    def reseed(self, seed: int, stream=None):
        self.seed = int(seed)
        _check("cse_reseed", lib().cse_reseed(self._h, self.seed, _stream(stream)))

    def profile(self, enable: bool, only: str = None):
        """cse_profile_enable; `only` names the one kernel group to time (cse_profile_only)."""
        _check("cse_profile_only", lib().cse_profile_only(self._h, only.encode() if only else None))
        _check("cse_profile_enable", lib().cse_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self):
        """{kernel name: (launches, total ms)} since the last read (synchronises)."""
        n = 16
        names = (C.c_char_p * n)()
        cnt = (C.c_int64 * n)()
        ms = (C.c_double * n)()
        m = lib().cse_profile_read(self._h, names, cnt, ms, n)
        if m < 0:
            raise CseError("cse_profile_read", m)
        return {names[i].decode(): (int(cnt[i]), float(ms[i])) for i in range(min(m, n))}

    def autotune(self, tiles: DeviceTiles, lam: float, alpha: float, stream=None):
        """cse_autotune: pick the simulation kernel's (threads per block, tiles per
        block) for this tile set; returns the pair."""
        n, g = C.c_int32(), C.c_int32()
        _check("cse_autotune", lib().cse_autotune(self._h, C.byref(tiles.struct), float(lam), float(alpha),
                                                  C.byref(n), C.byref(g), _stream(stream)))
        return n.value, g.value

    def set_option(self, option: int, value: int):
        _check("cse_set_option", lib().cse_set_option(self._h, int(option), int(value)))

    def statistics(self, tiles: DeviceTiles, stream=None):
        """Per-sim statistics: list of float32 tensors (one per tile, length K_i)."""
        K64 = tiles.K.to(torch.int64)
        off = torch.zeros_like(K64)
        off[1:] = torch.cumsum(K64, 0)[:-1]
        total = int(K64.sum().item())
        S = torch.empty(total, dtype=torch.float32, device=tiles.K.device)
        _check("cse_statistics", lib().cse_statistics(self._h, C.byref(tiles.struct), _ptr(off), _ptr(S),
                                                      _stream(stream)))
        return S, off

    def sync(self, stream=None):
        _check("cse_sync", lib().cse_sync(self._h, _stream(stream)))

    def _alloc(self, tiles, *shapes):
        dev = tiles.K.device
        return [torch.empty(s, dtype=dt, device=dev) for s, dt in shapes]

    def simulate_tiles(self, tiles: DeviceTiles, lam: float, stream=None):
        n, d = tiles.n_tiles, tiles.d
        R, X, G = self._alloc(tiles, ((n,), torch.int64), ((n, d), torch.int64), ((n, d), torch.float64))
        _check("cse_simulate_tiles", lib().cse_simulate_tiles(
            self._h, C.byref(tiles.struct), float(lam), _ptr(R), _ptr(X), _ptr(G), _stream(stream)))
        return R, X, G

    def type1_error(self, theta: torch.Tensor, null_mask, K, lam: float, stream=None):
        """cse_type1_error at the rows of theta [n, d] (device, float64, contiguous):
        returns (f_hat, R, score, K) with f_hat = R / K computed by the library.
        null_mask and K: per-point device tensors or ints (copied from the host)."""
        if theta.dtype != torch.float64 or not theta.is_contiguous() or theta.dim() != 2:
            raise TypeError("theta must be a contiguous float64 [n, d] tensor")
        n, d = theta.shape
        dev = theta.device
        nm = _per_point(null_mask, n, np.uint32, torch.int32, dev)
        Kt = _per_point(K, n, np.int32, torch.int32, dev)
        K_max = int(K) if not isinstance(K, torch.Tensor) else self.K_max   # per-point K: the context's bound
        fhat = torch.empty(n, dtype=torch.float64, device=dev)
        R = torch.empty(n, dtype=torch.int64, device=dev)
        G = torch.empty((n, d), dtype=torch.float64, device=dev)
        _check("cse_type1_error", lib().cse_type1_error(
            self._h, n, _ptr(theta), _ptr(nm), _ptr(Kt), K_max, float(lam), _ptr(fhat), _ptr(R), None, _ptr(G),
            _stream(stream)))
        return fhat, R, G, Kt

    def validate(self, tiles: DeviceTiles, lam: float, delta: float, stream=None):
        n, d = tiles.n_tiles, tiles.d
        R, X, G = self._alloc(tiles, ((n,), torch.int64), ((n, d), torch.int64), ((n, d), torch.float64))
        u0, b, q = self._alloc(tiles, ((n,), torch.float64), ((n,), torch.float64), ((n,), torch.float64))
        _check("cse_validate", lib().cse_validate(
            self._h, C.byref(tiles.struct), float(lam), float(delta), _ptr(R), _ptr(X), _ptr(G),
            _ptr(u0), _ptr(b), _ptr(q), _stream(stream)))
        return dict(R=R, Xrej=X, score=G, u0=u0, bound=b, qstar=q)

    def validate_lower(self, tiles: DeviceTiles, lam: float, delta: float, stream=None):
        n, d = tiles.n_tiles, tiles.d
        R, X, G = self._alloc(tiles, ((n,), torch.int64), ((n, d), torch.int64), ((n, d), torch.float64))
        l0, lo, q = self._alloc(tiles, ((n,), torch.float64), ((n,), torch.float64), ((n,), torch.float64))
        _check("cse_validate_lower", lib().cse_validate_lower(
            self._h, C.byref(tiles.struct), float(lam), float(delta), _ptr(R), _ptr(X), _ptr(G),
            _ptr(l0), _ptr(lo), _ptr(q), _stream(stream)))
        return dict(R=R, Xrej=X, score=G, l0=l0, lower=lo, qstar=q)

    def validate_band(self, tiles: DeviceTiles, lam: float, delta: float, stream=None):
        n, d = tiles.n_tiles, tiles.d
        R, X, G = self._alloc(tiles, ((n,), torch.int64), ((n, d), torch.int64), ((n, d), torch.float64))
        l0, lo, u0, up = self._alloc(tiles, *[((n,), torch.float64)] * 4)
        _check("cse_validate_band", lib().cse_validate_band(
            self._h, C.byref(tiles.struct), float(lam), float(delta), _ptr(R), _ptr(X), _ptr(G),
            _ptr(l0), _ptr(lo), _ptr(u0), _ptr(up), _stream(stream)))
        return dict(R=R, Xrej=X, score=G, l0=l0, lower=lo, u0=u0, upper=up)

    def validate_rand(self, tiles: DeviceTiles, lam: float, c: int, delta: float, stream=None):
        """cse_validate_rand: reject iff S < lam, or S == lam and the sim's tie-break word < c."""
        n, d = tiles.n_tiles, tiles.d
        R, X, G = self._alloc(tiles, ((n,), torch.int64), ((n, d), torch.int64), ((n, d), torch.float64))
        u0, b, q = self._alloc(tiles, ((n,), torch.float64), ((n,), torch.float64), ((n,), torch.float64))
        _check("cse_validate_rand", lib().cse_validate_rand(
            self._h, C.byref(tiles.struct), float(lam), int(c) & 0xFFFFFFFF, float(delta), _ptr(R), _ptr(X),
            _ptr(G), _ptr(u0), _ptr(b), _ptr(q), _stream(stream)))
        return dict(R=R, Xrej=X, score=G, u0=u0, bound=b, qstar=q)

    def calibrate_rand(self, tiles: DeviceTiles, alpha: float, stream=None):
        """cse_calibrate_rand: per-tile (lambda_i, c_i) and their lexicographic minimum.
        c_tile holds the uint32 words in an int32 tensor (view it as uint32)."""
        n = tiles.n_tiles
        ap, lt = self._alloc(tiles, ((n,), torch.float64), ((n,), torch.float64))
        (ct,) = self._alloc(tiles, ((n,), torch.int32))
        lam, cs = C.c_double(), C.c_uint32()
        _check("cse_calibrate_rand", lib().cse_calibrate_rand(
            self._h, C.byref(tiles.struct), float(alpha), _ptr(ap), _ptr(lt), _ptr(ct), C.byref(lam), C.byref(cs),
            _stream(stream)))
        return dict(alpha_prime=ap, lambda_tile=lt, c_tile=ct, lam=lam.value, c=int(cs.value))

    def calibrate(self, tiles: DeviceTiles, alpha: float, stream=None):
        n = tiles.n_tiles
        ap, lt = self._alloc(tiles, ((n,), torch.float64), ((n,), torch.float64))
        lam = C.c_double()
        _check("cse_calibrate", lib().cse_calibrate(
            self._h, C.byref(tiles.struct), float(alpha), _ptr(ap), _ptr(lt), C.byref(lam), _stream(stream)))
        return dict(alpha_prime=ap, lambda_tile=lt, lam=lam.value)

    def step_buffers(self, tiles: DeviceTiles):
        n, d = tiles.n_tiles, tiles.d
        names = ["R", "Xrej", "score", "u0", "bound", "qstar", "alpha_prime", "lambda_tile", "lam"]
        shapes = [((n,), torch.int64), ((n, d), torch.int64), ((n, d), torch.float64)] + \
                 [((n,), torch.float64)] * 5 + [((1,), torch.float64)]
        return dict(zip(names, self._alloc(tiles, *shapes)))

    def step(self, tiles: DeviceTiles, lam: float, delta: float, alpha: float, out=None, stream=None):
        out = out if out is not None else self.step_buffers(tiles)
        _check("cse_step", lib().cse_step(
            self._h, C.byref(tiles.struct), float(lam), float(delta), float(alpha),
            _ptr(out["R"]), _ptr(out["Xrej"]), _ptr(out["score"]), _ptr(out["u0"]), _ptr(out["bound"]),
            _ptr(out["qstar"]), _ptr(out["alpha_prime"]), _ptr(out["lambda_tile"]), _ptr(out["lam"]),
            _stream(stream)))
        return out


def simulate_tiles_static(design: W.Design, seed: int, tiles: DeviceTiles, lam: float, stream=None):
    """cse_simulate_tiles_static: the allocation-free simulation (outputs are
    allocated here by torch; the library itself allocates nothing)."""
    n, d = tiles.n_tiles, tiles.d
    dev = tiles.K.device
    R = torch.empty(n, dtype=torch.int64, device=dev)
    X = torch.empty((n, d), dtype=torch.int64, device=dev)
    G = torch.empty((n, d), dtype=torch.float64, device=dev)
    D = make_design(design)
    _check("cse_simulate_tiles_static", lib().cse_simulate_tiles_static(
        C.byref(D), int(seed), C.byref(tiles.struct), float(lam), _ptr(R), _ptr(X), _ptr(G), _stream(stream)))
    return R, X, G


PROBE_KINDS = {"alu": 0, "fma": 1, "dfma": 2, "smem_atomic": 3}


def probe_peak(kind: str, blocks_per_sm: int = 4, iters: int = 4096, reps: int = 5, stream=None):
    """cse_probe_peak: (lane-ops per second, ms per launch) of one pipe's probe."""
    ops, ms = C.c_double(), C.c_double()
    _check("cse_probe_peak", lib().cse_probe_peak(PROBE_KINDS[kind], int(blocks_per_sm), int(iters), int(reps),
                                                  C.byref(ops), C.byref(ms), _stream(stream)))
    return ops.value, ms.value


def score_backward(grad_out, score, K, stream=None):
    n, d = score.shape
    out = torch.empty_like(score)
    _check("cse_score_backward", lib().cse_score_backward(
        n, d, _ptr(grad_out.contiguous()), _ptr(score), _ptr(K), _ptr(out), _stream(stream)))
    return out


class StepGraph:
    """One whole step (cse_reseed + cse_step + cse_score_backward) captured in a
    CUDA graph and replayed: a single launch per step from the host.

    The context's scratch is sized by one direct call before capture (nothing
    may be allocated during capture); the seed, thresholds and outputs are the
    ones given here and are fixed in the graph.  The profiler must be off."""

    def __init__(self, ctx: "Context", tiles: DeviceTiles, lam: float, delta: float, alpha: float,
                 seed: int, out: dict, grad_out: torch.Tensor):
        self.ctx, self.tiles, self.out = ctx, tiles, out
        ctx.reseed(seed)
        ctx.step(tiles, lam, delta, alpha, out)
        score_backward(grad_out, out["score"], tiles.K)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(self.graph, stream=side):
            ctx.reseed(seed)
            ctx.step(tiles, lam, delta, alpha, out)
            self.grad = score_backward(grad_out, out["score"], tiles.K)
        torch.cuda.current_stream().wait_stream(side)

    def replay(self):
        self.graph.replay()
        return self.out, self.grad


class TypeIError(torch.autograd.Function):
    """Monte Carlo Type I Error f_hat(theta_i) = R_i / K_i at each point theta_i.

    Backward is the score-function adjoint (cse_score_backward):
    d f_hat_i / d theta_ia = score_ia / K_i with score = sum_k 1{rej}(T - grad A).

    Forward is one library call (cse_type1_error: the points' distinct
    coordinates are gathered on the device, then simulated); null_mask and K
    are per-point device tensors (uint32/int32) or plain ints for every point.
    """

    @staticmethod
    def forward(ctx_, theta, cse_ctx, null_mask, K, lam):
        fhat, R, G, Kt = cse_ctx.type1_error(theta.detach(), null_mask, K, lam)
        ctx_.save_for_backward(G, Kt)
        return fhat

    @staticmethod
    def backward(ctx_, grad_out):
        G, K = ctx_.saved_tensors
        if grad_out.dtype != torch.float64:
            raise TypeError("TypeIError: the incoming gradient must be float64")
        g = score_backward(grad_out.contiguous(), G, K)
        return g, None, None, None, None
