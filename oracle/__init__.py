"""FP64 CPU oracle for rejection sampling of the truncated-KdV Gibbs measure.

TEST INFRASTRUCTURE ONLY.  tests/, ``__graft_entry__.smoke()`` and the CPU
baseline / reference leg of ``bench.py`` are the only code allowed to import
this package.  The CUDA library and its binding never import it, and the two
share no code: they meet only through their inputs (parameters, seeds,
proposal indices).

The arithmetic lives in ``oracle.c`` (plain C, FP64, pthreads over proposals);
this module compiles it with gcc on first use and wraps it with ctypes.  The
learned-proposal oracle (MLP forward/backward in FP64) is in ``oracle.mlp``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

KMAX = 128
HIST_BINS = 256
N_EXCEED = 25
UNIFORM, PAPER, DIAG = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, FP64, no FMA contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Point(C.Structure):
    _fields_ = [("K", C.c_int), ("proposal", C.c_int), ("E0", C.c_double),
                ("beta_p", C.c_double), ("r", C.c_double), ("alpha", C.c_double),
                ("sigma2", C.c_double * KMAX), ("logM", C.c_double)]


class Rec(C.Structure):
    _fields_ = [("idx", C.c_uint64), ("lnU", C.c_double), ("logfg", C.c_double),
                ("delta", C.c_double), ("H2", C.c_double), ("H3", C.c_double),
                ("S", C.c_double), ("u0", C.c_double), ("accept", C.c_int),
                ("near", C.c_int), ("xhat", C.c_double * (2 * KMAX))]


class Stats(C.Structure):
    _fields_ = [("n_prop", C.c_uint64), ("n_acc", C.c_uint64), ("n_near", C.c_uint64),
                ("n_viol", C.c_uint64), ("max_delta", C.c_double), ("u_cap", C.c_double),
                ("sum_u0", C.c_double * 4), ("sum_grid", C.c_double * 4),
                ("spectrum", C.c_double * KMAX), ("hist", C.c_uint64 * HIST_BINS),
                ("exceed", C.c_uint64 * N_EXCEED)]


class SirStats(C.Structure):
    _fields_ = [("n_prop", C.c_uint64), ("n_kept", C.c_uint64), ("n_copies", C.c_uint64),
                ("sum_w", C.c_double), ("sum_w2", C.c_double), ("sum_wS", C.c_double),
                ("sum_w_u0", C.c_double * 4), ("sum_nS", C.c_double), ("sum_n_u0", C.c_double * 4),
                ("spectrum", C.c_double * KMAX)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            dp = C.POINTER(C.c_double)
            u32p = C.POINTER(C.c_uint32)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_uniform.argtypes = [C.c_uint32]
            L.orc_uniform.restype = C.c_double
            L.orc_uniform_ext.argtypes = [C.c_uint32, C.c_uint32, u32p, C.c_uint64, C.c_uint32]
            L.orc_uniform_ext.restype = C.c_double
            L.orc_box_muller.argtypes = [C.c_double, C.c_double, dp, dp]
            L.orc_stream.argtypes = [C.c_int, C.c_uint64, C.c_uint32, C.c_uint64, dp, dp]
            L.orc_tail_scan.argtypes = [C.c_int, C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint64, C.c_int,
                                        C.POINTER(C.c_uint64), C.c_uint64]
            L.orc_tail_scan.restype = C.c_uint64
            for f in ("orc_H2", "orc_H3_double", "orc_H3_triple"):
                getattr(L, f).argtypes = [C.c_int, C.c_double, dp]
                getattr(L, f).restype = C.c_double
            L.orc_H3_grid.argtypes = [C.c_int, C.c_double, dp, C.c_int]
            L.orc_H3_grid.restype = C.c_double
            L.orc_u_at.argtypes = [C.c_int, C.c_double, dp, C.c_double]
            L.orc_u_at.restype = C.c_double
            L.orc_F_alpha.argtypes = [C.c_int, C.c_double, C.c_double]
            L.orc_F_alpha.restype = C.c_double
            L.orc_alpha_star.argtypes = [C.c_int, C.c_double]
            L.orc_alpha_star.restype = C.c_double
            L.orc_point_init.argtypes = [C.POINTER(Point), C.c_int, C.c_double, C.c_double,
                                         C.c_double, C.c_int]
            L.orc_point_init.restype = C.c_int
            L.orc_log_fg.argtypes = [C.POINTER(Point), dp]
            L.orc_log_fg.restype = C.c_double
            L.orc_log_M.argtypes = [C.POINTER(Point), C.c_int, C.c_uint64, dp]
            L.orc_log_M.restype = C.c_double
            L.orc_nelder_mead.argtypes = [C.POINTER(Point), dp, dp, C.c_long]
            L.orc_nelder_mead.restype = C.c_double
            L.orc_replay.argtypes = [C.POINTER(Point), C.c_uint64, C.c_uint32,
                                     C.POINTER(C.c_uint64), C.c_uint64, C.c_int, C.POINTER(Rec)]
            L.orc_run_stats.argtypes = [C.POINTER(Point), C.c_uint64, C.c_uint32, C.c_uint64,
                                        C.c_uint64, C.c_int, C.POINTER(Stats)]
            L.orc_run_accepted.argtypes = [C.POINTER(Point), C.c_uint64, C.c_uint32, C.c_uint64,
                                           C.c_uint64, C.c_int, C.POINTER(Rec), C.c_uint64]
            L.orc_run_accepted.restype = C.c_uint64
            L.orc_poisson_tail.argtypes = [C.c_double, C.c_int]
            L.orc_poisson_tail.restype = C.c_double
            L.orc_poisson_count.argtypes = [C.c_double, C.c_double]
            L.orc_poisson_count.restype = C.c_int
            L.orc_run_sir.argtypes = [C.POINTER(Point), C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint64, C.c_double,
                                      C.c_int, C.POINTER(SirStats), C.POINTER(Rec), C.POINTER(C.c_uint32),
                                      C.c_uint64]
            L.orc_run_sir.restype = C.c_uint64
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _vec(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


# ------------------------------------------------------------------ stream
def philox(ctr, key):
    """Philox4x32-10 block for counter (4 words) and key (2 words)."""
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniform(w):
    return lib().orc_uniform(int(w) & 0xFFFFFFFF)


def uniform_ext(w, g, seed, idx, point_id):
    """Uniform of word w at stream position g of proposal idx, lowest bucket refined."""
    k = (C.c_uint32 * 2)(seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return lib().orc_uniform_ext(int(w) & 0xFFFFFFFF, int(g), k, int(idx), int(point_id) & 0xFFFFFFFF)


def tail_scan(K, seed, point_id, idx0, n, which=3, cap=1 << 16):
    """Indices of [idx0, idx0+n) with a radius (which & 1) or accept (which & 2)
    word in the lowest bucket of the uniform map; returns (indices, total)."""
    out = np.zeros(cap, dtype=np.uint64)
    tot = lib().orc_tail_scan(K, seed, point_id, idx0, n, which, out.ctypes.data_as(C.POINTER(C.c_uint64)), cap)
    return out[:min(tot, cap)], int(tot)


def box_muller(u1, u2):
    a, b = C.c_double(), C.c_double()
    lib().orc_box_muller(float(u1), float(u2), C.byref(a), C.byref(b))
    return a.value, b.value


def stream(K, seed, point_id, idx):
    """(z[2K] in [cos | sin] layout, accept uniform) of proposal idx."""
    z = np.zeros(2 * K)
    u = C.c_double()
    lib().orc_stream(K, seed, point_id, idx, _dp(z), C.byref(u))
    return z, u.value


# --------------------------------------------------------------- Hamiltonian
def H2(K, E0, xh):
    xh = _vec(xh)
    return lib().orc_H2(K, E0, _dp(xh))


def H3_double(K, E0, xh):
    xh = _vec(xh)
    return lib().orc_H3_double(K, E0, _dp(xh))


def H3_triple(K, E0, xh):
    xh = _vec(xh)
    return lib().orc_H3_triple(K, E0, _dp(xh))


def H3_grid(K, E0, xh, N):
    xh = _vec(xh)
    return lib().orc_H3_grid(K, E0, _dp(xh), N)


def u_at(K, E0, xh, xi):
    xh = _vec(xh)
    return lib().orc_u_at(K, E0, _dp(xh), xi)


# ----------------------------------------------------------------- proposal
def F_alpha(K, beta_p, alpha):
    return lib().orc_F_alpha(K, beta_p, alpha)


def alpha_star(K, beta_p):
    return lib().orc_alpha_star(K, beta_p)


def make_point(K, E0, beta_p, r, proposal, sigma2=None, logM=None):
    """Parameter point.  proposal: UNIFORM, PAPER (alpha* from Eq. 29) or DIAG
    (explicit pair variances sigma2[k-1], k = 1..K)."""
    pt = Point()
    init_prop = PAPER if proposal == PAPER else UNIFORM
    rc = lib().orc_point_init(C.byref(pt), K, E0, beta_p, r, init_prop)
    if rc != 0:
        raise ValueError("no alpha* root: beta' >= K^2 sum 1/k^2")
    if proposal == DIAG:
        pt.proposal = DIAG
        s2 = _vec(sigma2)
        assert s2.shape == (K,)
        for k in range(K):
            pt.sigma2[k] = float(s2[k])
    if logM is not None:
        pt.logM = float(logM)
    return pt


def log_fg(pt, xh):
    xh = _vec(xh)
    return lib().orc_log_fg(C.byref(pt), _dp(xh))


def log_M(pt, n_random_starts=4, seed=12345, return_argmax=False):
    xb = np.zeros(2 * pt.K)
    v = lib().orc_log_M(C.byref(pt), n_random_starts, seed, _dp(xb))
    return (v, xb) if return_argmax else v


def nelder_mead(pt, xh0, max_evals=400000):
    x0 = _vec(xh0)
    xo = np.zeros(2 * pt.K)
    v = lib().orc_nelder_mead(C.byref(pt), _dp(x0), _dp(xo), max_evals)
    return v, xo


# ------------------------------------------------------------------ sampler
def _recs_to_dict(recs, n, K):
    out = {f: np.array([getattr(recs[i], f) for i in range(n)])
           for f in ("idx", "lnU", "logfg", "delta", "H2", "H3", "S", "u0", "accept", "near")}
    out["accept"] = out["accept"].astype(bool)
    out["near"] = out["near"].astype(bool)
    xh = np.zeros((n, 2 * K))
    for i in range(n):
        xh[i] = np.frombuffer(recs[i].xhat, dtype=np.float64, count=2 * K)
    out["xhat"] = xh
    return out


def replay(pt, seed, point_id, idx, nthreads=None):
    """Replay the listed proposal indices; returns a dict of per-proposal arrays."""
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64))
    n = int(idx.size)
    recs = (Rec * max(n, 1))()
    nt = nthreads or os.cpu_count() or 1
    lib().orc_replay(C.byref(pt), seed, point_id, idx.ctypes.data_as(C.POINTER(C.c_uint64)),
                     n, nt, recs)
    return _recs_to_dict(recs, n, pt.K)


def run_stats(pt, seed, point_id, idx0, n, nthreads=None):
    st = Stats()
    nt = nthreads or os.cpu_count() or 1
    lib().orc_run_stats(C.byref(pt), seed, point_id, idx0, n, nt, C.byref(st))
    d = {"n_prop": st.n_prop, "n_acc": st.n_acc, "n_near": st.n_near, "n_viol": st.n_viol,
         "max_delta": st.max_delta, "u_cap": st.u_cap,
         "sum_u0": np.array(st.sum_u0[:]), "sum_grid": np.array(st.sum_grid[:]),
         "spectrum": np.array(st.spectrum[:pt.K]),
         "hist": np.array(st.hist[:], dtype=np.uint64),
         "exceed": np.array(st.exceed[:], dtype=np.uint64), "nthreads": nt}
    return d


def run_accepted(pt, seed, point_id, idx0, n, cap=1 << 16, nthreads=None):
    recs = (Rec * max(cap, 1))()
    nt = nthreads or os.cpu_count() or 1
    total = lib().orc_run_accepted(C.byref(pt), seed, point_id, idx0, n, nt, recs, cap)
    got = min(int(total), cap)
    return int(total), _recs_to_dict(recs, got, pt.K)


def moments(n, sums):
    """mean, variance, skewness, kurtosis from n and raw power sums s1..s4."""
    if n == 0:
        return dict(mean=float("nan"), var=float("nan"), skew=float("nan"), kurt=float("nan"))
    m1, m2, m3, m4 = (s / n for s in sums)
    var = m2 - m1 * m1
    c3 = m3 - 3 * m1 * m2 + 2 * m1 ** 3
    c4 = m4 - 4 * m1 * m3 + 6 * m1 * m1 * m2 - 3 * m1 ** 4
    return dict(mean=m1, var=var, skew=c3 / var ** 1.5, kurt=c4 / var ** 2)


# ------------------------------------------------------------------ SIR
def poisson_tail(lam, k):
    """P(N >= k), N ~ Poisson(lam)."""
    return lib().orc_poisson_tail(float(lam), int(k))


def poisson_count(lam, u):
    """#{k >= 1 : u < P(N >= k)}: a Poisson(lam) count by inversion of u."""
    return lib().orc_poisson_count(float(lam), float(u))


def run_sir(pt, seed, point_id, idx0, n, c, cap=1 << 16, nthreads=None):
    """SIR with Poisson copy numbers n_i ~ Poisson(c exp(Delta_i)) over proposals
    idx0 .. idx0+n-1: returns (statistics dict, kept records dict with "copies")."""
    st = SirStats()
    recs = (Rec * max(cap, 1))()
    cnt = (C.c_uint32 * max(cap, 1))()
    nt = nthreads or os.cpu_count() or 1
    total = lib().orc_run_sir(C.byref(pt), seed, point_id, idx0, n, float(c), nt, C.byref(st), recs, cnt, cap)
    got = min(total, cap)
    d = {"n_prop": st.n_prop, "n_kept": st.n_kept, "n_copies": st.n_copies, "sum_w": st.sum_w,
         "sum_w2": st.sum_w2, "sum_wS": st.sum_wS, "sum_w_u0": np.array(st.sum_w_u0[:]), "sum_nS": st.sum_nS,
         "sum_n_u0": np.array(st.sum_n_u0[:]), "spectrum": np.array(st.spectrum[:pt.K])}
    kept = _recs_to_dict(recs, got, pt.K)
    kept["copies"] = np.array(cnt[:got], dtype=np.int64)
    return d, kept
