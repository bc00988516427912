"""GB300 (sm_103a) rejection sampler for the truncated-KdV Gibbs measure.

Python binding of the C ABI in include/tkdv.h (argument marshalling only:
every step of the sampler runs in the library's CUDA kernels).  The functions
carry the C names (``sampler_create``, ``sampler_run``, ``sampler_stats`` ...);
:class:`Sampler` wraps one handle.  PyTorch is used only to hand the library a
CUDA stream (``torch.cuda.current_stream()``) and device buffers for records.

The shared library is built by ``__graft_entry__.build()`` (or
``paper_2411_16952_gb300._build.build()``).  There is no fallback: if
libtkdv.so is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtkdv.so")

TKDV_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "NO_ALPHA", -3: "CUDA", -4: "OOM", -5: "TIMEOUT",
          -6: "UNSUPPORTED", -7: "ENVELOPE", -8: "TOO_LARGE"}
STATIC_MAX_PROPOSALS = 262144
PROPOSAL_UNIFORM, PROPOSAL_PAPER, PROPOSAL_LEARNED = 0, 1, 2
H3_TRIAD_F32, H3_GRID_BF16X3, H3_AUTO = 0, 1, 2
MAX_POINTS = 64
HIST_BINS = 256
N_EXCEED = 25
KMAX = 128

EXPORTED = ["tkdv_record_bytes", "sampler_create", "sampler_create_ex", "sampler_run",
            "sampler_run_budgets", "sampler_run_ranges", "sampler_stats", "sampler_samples",
            "sampler_reset", "sampler_sync", "sampler_set_deadline_ns", "sampler_point_info",
            "sampler_replay", "sampler_autotune", "sampler_launch_config", "sampler_last_error",
            "sampler_destroy", "tkdv_alpha_star", "tkdv_log_M", "sampler_run_static",
            "sampler_set_trace", "tkdv_check_radius_error", "tkdv_check_radius_error_log",
            "sampler_h3_form", "sampler_batch_run", "sampler_set_launch", "tkdv_mlp_create", "tkdv_mlp_destroy", "tkdv_mlp_last_error",
            "tkdv_mlp_features", "tkdv_mlp_get_params", "tkdv_mlp_set_params", "tkdv_mlp_infer",
            "tkdv_mlp_set_data", "tkdv_mlp_set_data_records", "tkdv_mlp_rows", "tkdv_mlp_step"]
MLP_NPARAM = 8640


class TkdvError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class tkdv_point(C.Structure):
    _fields_ = [("beta_p", C.c_double), ("E0", C.c_double), ("r", C.c_double),
                ("proposal", C.c_int), ("point_id", C.c_uint32), ("override_logM", C.c_int),
                ("logM", C.c_double), ("log_var_correction", C.POINTER(C.c_double)), ("sir_c", C.c_double)]


class tkdv_options(C.Structure):
    _fields_ = [("K", C.c_int), ("h3_mode", C.c_int), ("grid_N", C.c_int),
                ("sample_capacity", C.c_uint64), ("cuda_stream", C.c_void_p),
                ("use_graph", C.c_int), ("ctas_per_sm", C.c_int), ("threads_per_cta", C.c_int), ("sir", C.c_int)]


class tkdv_stats(C.Structure):
    _fields_ = [("n_proposals", C.c_uint64), ("n_accepted", C.c_uint64),
                ("n_near_threshold", C.c_uint64), ("n_refined", C.c_uint64),
                ("n_envelope_violations", C.c_uint64), ("n_dropped", C.c_uint64),
                ("n_fallback", C.c_uint64), ("max_delta", C.c_double), ("logM", C.c_double),
                ("alpha_star", C.c_double), ("sum_u0", C.c_double * 4), ("mean", C.c_double),
                ("var", C.c_double), ("skew", C.c_double), ("kurt", C.c_double),
                ("hist", C.c_uint64 * HIST_BINS), ("hist_lo", C.c_double), ("hist_hi", C.c_double),
                ("exceed", C.c_uint64 * N_EXCEED), ("spectrum", C.c_double * KMAX), ("n_kept", C.c_uint64),
                ("sir_sum_w", C.c_double), ("sir_sum_w2", C.c_double), ("sir_sum_wS", C.c_double),
                ("sir_sum_w_u0", C.c_double * 4)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libtkdv.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libtkdv.so is not built; run __graft_entry__.build() first")
            L = C.CDLL(LIB_PATH)
            vp, u64, i, d = C.c_void_p, C.c_uint64, C.c_int, C.c_double
            dp, u64p = C.POINTER(C.c_double), C.POINTER(C.c_uint64)
            L.tkdv_record_bytes.argtypes = [i]
            L.tkdv_record_bytes.restype = C.c_size_t
            L.sampler_create.argtypes = [i, d, d, d, i, C.POINTER(vp)]
            L.sampler_create_ex.argtypes = [C.POINTER(tkdv_point), i, C.POINTER(tkdv_options),
                                            C.POINTER(vp)]
            L.sampler_run.argtypes = [vp, u64, u64]
            L.sampler_run_budgets.argtypes = [vp, u64p, u64]
            L.sampler_run_ranges.argtypes = [vp, u64p, u64p, u64]
            L.sampler_stats.argtypes = [vp, C.POINTER(tkdv_stats), i]
            L.sampler_samples.argtypes = [vp, vp, i, u64, u64p]
            L.sampler_reset.argtypes = [vp]
            L.sampler_sync.argtypes = [vp]
            L.sampler_set_deadline_ns.argtypes = [vp, u64]
            L.sampler_set_trace.argtypes = [vp, vp, u64]
            fp, ip = C.POINTER(C.c_float), C.POINTER(C.c_int)
            L.tkdv_mlp_create.argtypes = [u64, C.POINTER(vp)]
            L.tkdv_mlp_destroy.argtypes = [vp]
            L.tkdv_mlp_destroy.restype = None
            L.tkdv_mlp_last_error.argtypes = [vp]
            L.tkdv_mlp_last_error.restype = C.c_char_p
            L.tkdv_mlp_features.argtypes = [i, d, d, d, dp]
            L.tkdv_mlp_get_params.argtypes = [vp, fp, fp]
            L.tkdv_mlp_set_params.argtypes = [vp, fp]
            L.tkdv_mlp_infer.argtypes = [vp, i, dp, ip, dp]
            L.tkdv_mlp_set_data.argtypes = [vp, i, ip, dp, dp, u64p, fp, fp]
            L.tkdv_mlp_set_data_records.argtypes = [vp, i, ip, dp, dp, dp, vp, u64, i, u64]
            L.tkdv_mlp_rows.argtypes = [vp, u64p]
            L.tkdv_mlp_step.argtypes = [vp, C.c_float, C.c_float, i, dp, fp]
            L.sampler_point_info.argtypes = [vp, i, dp, dp, dp]
            L.sampler_replay.argtypes = [vp, i, u64p, u64, u64, dp]
            L.sampler_autotune.argtypes = [vp, u64, dp]
            L.sampler_launch_config.argtypes = [vp, C.POINTER(i), C.POINTER(i), C.POINTER(C.c_uint32)]
            L.sampler_h3_form.argtypes = [vp]
            L.sampler_set_launch.argtypes = [vp, i, i]
            L.sampler_batch_run.argtypes = [C.POINTER(tkdv_point), i, C.POINTER(tkdv_options), u64p, u64,
                                            C.POINTER(tkdv_stats)]
            L.sampler_last_error.argtypes = [vp]
            L.sampler_last_error.restype = C.c_char_p
            L.sampler_destroy.argtypes = [vp]
            L.sampler_destroy.restype = None
            L.tkdv_alpha_star.argtypes = [i, d, dp]
            L.tkdv_log_M.argtypes = [i, d, d, d, dp, dp]
            L.tkdv_check_radius_error.argtypes = [dp, C.POINTER(C.c_uint32)]
            L.tkdv_check_radius_error_log.argtypes = [dp, C.POINTER(C.c_uint32)]
            L.sampler_field_maxima.argtypes = [vp, u64, dp, C.POINTER(C.c_int32), u64p]
            L.sampler_run_static.argtypes = [i, C.POINTER(tkdv_point), u64, u64, u64, vp, u64, u64p,
                                             C.POINTER(tkdv_stats), vp]
            _lib = L
    return _lib


def _check(rc, handle=None):
    if rc != TKDV_OK:
        msg = lib().sampler_last_error(handle)
        raise TkdvError(rc, msg.decode() if msg else "")


# ---- the C entry points under their own names ------------------------------
def tkdv_record_bytes(K):
    return int(lib().tkdv_record_bytes(K))


def sampler_field_maxima(h, max_records):
    """(umax, j) of the first kept records on the 2K-point grid xi_j = -pi + pi j/K."""
    umax = np.zeros(max(int(max_records), 1))
    jm = np.zeros(max(int(max_records), 1), dtype=np.int32)
    n = C.c_uint64()
    _check(lib().sampler_field_maxima(h, max_records, _dptr(umax), jm.ctypes.data_as(C.POINTER(C.c_int32)),
                                      C.byref(n)), h)
    return umax[:n.value], jm[:n.value]


def tkdv_check_radius_error():
    """(largest ratio of error to its bound 2^-21 + 2^-21 rho, a word attaining
    it) of the fast path's FP32 radius -2 ln u over all 2^23 values of the
    uniform map (runs on the device)."""
    err, w = C.c_double(), C.c_uint32()
    _check(lib().tkdv_check_radius_error(C.byref(err), C.byref(w)))
    return err.value, w.value


def tkdv_check_radius_error_log():
    """The same for the warp form's radius -2 logf(u) (K > 64) against its
    purely relative bound 2^-22 rho."""
    err, w = C.c_double(), C.c_uint32()
    _check(lib().tkdv_check_radius_error_log(C.byref(err), C.byref(w)))
    return err.value, w.value


def tkdv_alpha_star(K, beta_p):
    out = C.c_double()
    _check(lib().tkdv_alpha_star(K, beta_p, C.byref(out)))
    return out.value


def tkdv_log_M(K, beta_p, E0, r, sigma2=None):
    out = C.c_double()
    s2 = None
    if sigma2 is not None:
        arr = np.ascontiguousarray(np.asarray(sigma2, dtype=np.float64))
        s2 = arr.ctypes.data_as(C.POINTER(C.c_double))
    _check(lib().tkdv_log_M(K, beta_p, E0, r, s2, C.byref(out)))
    return out.value


def sampler_create(K, beta_p, E0, r, proposal):
    h = C.c_void_p()
    _check(lib().sampler_create(K, beta_p, E0, r, proposal, C.byref(h)))
    return h


def sampler_create_ex(points, options):
    arr = (tkdv_point * len(points))(*points)
    h = C.c_void_p()
    _check(lib().sampler_create_ex(arr, len(points), C.byref(options), C.byref(h)))
    return h


def sampler_run(h, n_proposals, seed):
    _check(lib().sampler_run(h, n_proposals, seed), h)


def sampler_run_budgets(h, budgets, seed):
    b = np.ascontiguousarray(np.asarray(budgets, dtype=np.uint64))
    _check(lib().sampler_run_budgets(h, b.ctypes.data_as(C.POINTER(C.c_uint64)), seed), h)


def sampler_run_ranges(h, idx0, count, seed):
    a = np.ascontiguousarray(np.asarray(idx0, dtype=np.uint64))
    b = np.ascontiguousarray(np.asarray(count, dtype=np.uint64))
    _check(lib().sampler_run_ranges(h, a.ctypes.data_as(C.POINTER(C.c_uint64)),
                                    b.ctypes.data_as(C.POINTER(C.c_uint64)), seed), h)


def sampler_stats(h, n_points):
    out = (tkdv_stats * n_points)()
    _check(lib().sampler_stats(h, out, n_points), h)
    return [_stats_dict(out[p]) for p in range(n_points)]


def sampler_samples(h, K, max_records, device_dst=None, host_dst=None):
    """Accepted records: a dict of numpy arrays (host), or, with device_dst (a
    torch uint8 CUDA tensor of max_records * record_bytes), the record count
    after a device-to-device copy into it, or, with host_dst (a caller-owned
    host buffer of at least max_records * record_bytes bytes: a torch uint8
    CPU tensor, pinned for full copy speed, or a numpy uint8 array), the
    record count after the raw records were copied into it (no decoding)."""
    n = C.c_uint64()
    rb = tkdv_record_bytes(K)
    if device_dst is not None:
        _check(lib().sampler_samples(h, C.c_void_p(device_dst.data_ptr()), 1, max_records,
                                     C.byref(n)), h)
        return int(n.value)
    if host_dst is not None:
        ptr = host_dst.data_ptr() if hasattr(host_dst, "data_ptr") else host_dst.ctypes.data
        nbytes = host_dst.numel() if hasattr(host_dst, "numel") else host_dst.nbytes
        if nbytes < max_records * rb:
            raise ValueError("host_dst holds %d bytes, %d records need %d" % (nbytes, max_records, max_records * rb))
        _check(lib().sampler_samples(h, C.c_void_p(ptr), 0, max_records, C.byref(n)), h)
        return int(n.value)
    buf = np.zeros(max(1, max_records) * rb, dtype=np.uint8)
    _check(lib().sampler_samples(h, buf.ctypes.data_as(C.c_void_p), 0, max_records, C.byref(n)), h)
    return decode_records(buf[: int(n.value) * rb], K)


def sampler_reset(h):
    _check(lib().sampler_reset(h), h)


def sampler_sync(h):
    _check(lib().sampler_sync(h), h)


def sampler_set_trace(h, dev_tensor, n):
    """Grid form: later runs write (log f/(Mg), T) of point 0's first n proposals
    into dev_tensor (a float32 CUDA tensor of 2n elements, or None to stop)."""
    ptr = C.c_void_p(dev_tensor.data_ptr()) if dev_tensor is not None else None
    _check(lib().sampler_set_trace(h, ptr, n if dev_tensor is not None else 0), h)


def sampler_set_deadline_ns(h, ns):
    _check(lib().sampler_set_deadline_ns(h, ns), h)


def sampler_point_info(h, p, K):
    a, lm = C.c_double(), C.c_double()
    s2 = np.zeros(K)
    _check(lib().sampler_point_info(h, p, C.byref(a), C.byref(lm),
                                    s2.ctypes.data_as(C.POINTER(C.c_double))), h)
    return a.value, lm.value, s2


def sampler_replay(h, p, K, idx, seed):
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64))
    n = int(idx.size)
    out = np.zeros((max(n, 1), 8 + 2 * K))
    _check(lib().sampler_replay(h, p, idx.ctypes.data_as(C.POINTER(C.c_uint64)), n, seed,
                                out.ctypes.data_as(C.POINTER(C.c_double))), h)
    out = out[:n]
    return {"delta": out[:, 0], "lnU": out[:, 1], "accept": out[:, 2] > 0.5,
            "flags": out[:, 3].astype(np.int64), "H2": out[:, 4], "H3": out[:, 5],
            "u0": out[:, 6], "S": out[:, 7], "xhat": out[:, 8:]}


def sampler_autotune(h, calib_proposals):
    us = C.c_double()
    _check(lib().sampler_autotune(h, calib_proposals, C.byref(us)), h)
    return us.value


def sampler_set_launch(h, variant, ctas_per_sm=0):
    """Pin the launch shape of later runs (see include/tkdv.h)."""
    _check(lib().sampler_set_launch(h, variant, ctas_per_sm), h)


def sampler_h3_form(h):
    """H3 form of the next run: H3_TRIAD_F32 or H3_GRID_BF16X3."""
    f = lib().sampler_h3_form(h)
    _check(f if f < 0 else TKDV_OK, h)
    return f


def sampler_batch_run(points, options, budgets, seed):
    """One call for a batch of points (create, run the budgets from index 0,
    statistics, destroy): a list of statistics dicts."""
    arr = (tkdv_point * len(points))(*points)
    b = np.ascontiguousarray(np.asarray(budgets, dtype=np.uint64))
    if b.shape != (len(points),):
        raise ValueError("one budget per point")
    out = (tkdv_stats * len(points))()
    _check(lib().sampler_batch_run(arr, len(points), C.byref(options), b.ctypes.data_as(C.POINTER(C.c_uint64)),
                                   seed, out))
    return [_stats_dict(out[p]) for p in range(len(points))]


def sampler_launch_config(h):
    c, t, ch = C.c_int(), C.c_int(), C.c_uint32()
    _check(lib().sampler_launch_config(h, C.byref(c), C.byref(t), C.byref(ch)), h)
    return {"ctas": c.value, "threads": t.value, "chunk": ch.value}


def sampler_last_error(h=None):
    m = lib().sampler_last_error(h)
    return m.decode() if m else ""


def sampler_destroy(h):
    if h:
        lib().sampler_destroy(h)


def sampler_run_static(K, point, idx0, n_proposals, seed, records=None, capacity=0, stream=None):
    """One run that allocates nothing (see include/tkdv.h): for callers whose
    device memory is owned elsewhere or who must not call cudaMalloc.
    records: the caller's contiguous torch uint8 tensor on the current CUDA
    device, holding at least capacity * tkdv_record_bytes(K) bytes (or None
    with capacity 0); anything else raises TkdvError(INVALID_ARG) before the
    library is called.  Returns (stats dict, number of records written)."""
    st = tkdv_stats()
    nrec = C.c_uint64()
    if records is not None:
        # the kernels write up to `capacity` records into this buffer: it must
        # be a uint8 tensor on the current CUDA device holding them all
        import torch
        rb = tkdv_record_bytes(K)
        if not (isinstance(records, torch.Tensor) and records.is_cuda and records.dtype == torch.uint8
                and records.is_contiguous()):
            raise TkdvError(-1, "sampler_run_static: records must be a contiguous uint8 CUDA tensor")
        if records.device.index != torch.cuda.current_device():
            raise TkdvError(-1, "sampler_run_static: records are on cuda:%d, the current device is cuda:%d"
                            % (records.device.index, torch.cuda.current_device()))
        if capacity < 0 or capacity * rb > records.numel():
            raise TkdvError(-1, "sampler_run_static: %d records of %d bytes do not fit a buffer of %d bytes"
                            % (capacity, rb, records.numel()))
    elif capacity:
        raise TkdvError(-1, "sampler_run_static: capacity > 0 needs a records buffer")
    dst = C.c_void_p(records.data_ptr()) if records is not None else None
    s = None if stream is None else C.c_void_p(int(getattr(stream, "cuda_stream", stream)) or 1)
    rc = lib().sampler_run_static(K, C.byref(point), idx0, n_proposals, seed, dst,
                                  capacity if records is not None else 0, C.byref(nrec), C.byref(st), s)
    if rc != TKDV_OK:
        raise TkdvError(rc, "sampler_run_static")
    return _stats_dict(st), int(nrec.value)


# ---- learned proposal ------------------------------------------------------
def _mcheck(rc, m):
    if rc != TKDV_OK:
        msg = lib().tkdv_mlp_last_error(m)
        raise TkdvError(rc, msg.decode() if msg else "")


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def tkdv_mlp_create(seed=0):
    m = C.c_void_p()
    _check(lib().tkdv_mlp_create(seed, C.byref(m)))
    return m


def tkdv_mlp_destroy(m):
    if m:
        lib().tkdv_mlp_destroy(m)


def tkdv_mlp_last_error(m):
    s = lib().tkdv_mlp_last_error(m)
    return s.decode() if s else ""


def tkdv_mlp_features(K, beta_p, E0, r):
    out = np.zeros(4)
    _check(lib().tkdv_mlp_features(K, beta_p, E0, r, _dptr(out)))
    return out


def tkdv_mlp_get_params(m):
    master = np.zeros(MLP_NPARAM, dtype=np.float32)
    bf = np.zeros(MLP_NPARAM, dtype=np.float32)
    _mcheck(lib().tkdv_mlp_get_params(m, _fptr(master), _fptr(bf)), m)
    return master, bf


def tkdv_mlp_set_params(m, master):
    a = np.ascontiguousarray(np.asarray(master, dtype=np.float32))
    assert a.size == MLP_NPARAM
    _mcheck(lib().tkdv_mlp_set_params(m, _fptr(a)), m)


def tkdv_mlp_infer(m, feats, Ks):
    f = np.ascontiguousarray(np.asarray(feats, dtype=np.float64).reshape(-1, 4))
    P = f.shape[0]
    k = np.ascontiguousarray(np.asarray(Ks, dtype=np.int32))
    out = np.zeros((P, 64))
    _mcheck(lib().tkdv_mlp_infer(m, P, _dptr(f), k.ctypes.data_as(C.POINTER(C.c_int)), _dptr(out)), m)
    return out


def tkdv_mlp_set_data(m, Ks, feats, w_paper, s_list, z_list=None):
    """Training set from host arrays: s_list[p] is (n_p, K_p) pair energies."""
    P = len(Ks)
    k = np.ascontiguousarray(np.asarray(Ks, dtype=np.int32))
    f = np.ascontiguousarray(np.asarray(feats, dtype=np.float64).reshape(P, 4))
    wp = np.zeros((P, 64))
    for p in range(P):
        wp[p, :Ks[p]] = w_paper[p]
    stride = (max(Ks) + 3) // 4 * 4
    counts = np.array([len(s) for s in s_list], dtype=np.uint64)
    rows = np.zeros((int(counts.sum()), stride), dtype=np.float32)
    z = np.zeros(int(counts.sum()), dtype=np.float32)
    o = 0
    for p in range(P):
        n = len(s_list[p])
        rows[o:o + n, :Ks[p]] = s_list[p]
        if z_list is not None:
            z[o:o + n] = z_list[p]
        o += n
    _mcheck(lib().tkdv_mlp_set_data(m, P, k.ctypes.data_as(C.POINTER(C.c_int)), _dptr(f), _dptr(wp),
                                    counts.ctypes.data_as(C.POINTER(C.c_uint64)), _fptr(rows), _fptr(z)), m)


def tkdv_mlp_set_data_records(m, Ks, feats, w_paper, zcoef, records_dev, n_records, K_records, max_per_point):
    P = len(Ks)
    k = np.ascontiguousarray(np.asarray(Ks, dtype=np.int32))
    f = np.ascontiguousarray(np.asarray(feats, dtype=np.float64).reshape(P, 4))
    wp = np.zeros((P, 64))
    for p in range(P):
        wp[p, :Ks[p]] = w_paper[p]
    zc = np.ascontiguousarray(np.asarray(zcoef, dtype=np.float64).reshape(P, 2))
    _mcheck(lib().tkdv_mlp_set_data_records(m, P, k.ctypes.data_as(C.POINTER(C.c_int)), _dptr(f), _dptr(wp),
                                            _dptr(zc), C.c_void_p(records_dev.data_ptr()), n_records,
                                            K_records, max_per_point), m)


def tkdv_mlp_rows(m, P):
    c = np.zeros(P, dtype=np.uint64)
    _mcheck(lib().tkdv_mlp_rows(m, c.ctypes.data_as(C.POINTER(C.c_uint64))), m)
    return c


def tkdv_mlp_step(m, lr=1e-2, tau=0.0, update=True, want_grad=False):
    loss = C.c_double()
    g = np.zeros(MLP_NPARAM, dtype=np.float32) if want_grad else None
    _mcheck(lib().tkdv_mlp_step(m, lr, tau, 1 if update else 0, C.byref(loss),
                                _fptr(g) if want_grad else None), m)
    return (loss.value, g) if want_grad else loss.value


# ---- helpers ---------------------------------------------------------------
def _stats_dict(s):
    return {"n_proposals": s.n_proposals, "n_accepted": s.n_accepted,
            "n_near_threshold": s.n_near_threshold, "n_refined": s.n_refined,
            "n_envelope_violations": s.n_envelope_violations, "n_dropped": s.n_dropped,
            "n_fallback": s.n_fallback, "max_delta": s.max_delta, "logM": s.logM,
            "alpha_star": s.alpha_star, "sum_u0": np.array(s.sum_u0[:]), "mean": s.mean,
            "var": s.var, "skew": s.skew, "kurt": s.kurt,
            "hist": np.array(s.hist[:], dtype=np.uint64), "hist_lo": s.hist_lo,
            "hist_hi": s.hist_hi, "exceed": np.array(s.exceed[:], dtype=np.uint64),
            "spectrum": np.array(s.spectrum[:]), "n_kept": s.n_kept, "sir_sum_w": s.sir_sum_w,
            "sir_sum_w2": s.sir_sum_w2, "sir_sum_wS": s.sir_sum_wS, "sir_sum_w_u0": np.array(s.sir_sum_w_u0[:])}


def decode_records(buf, K):
    rb = tkdv_record_bytes(K)
    n = len(buf) // rb
    raw = np.frombuffer(bytes(buf), dtype=np.uint8).reshape(n, rb) if n else np.zeros((0, rb), np.uint8)
    return {"idx": raw[:, 0:8].copy().view(np.uint64).reshape(n),
            "point": raw[:, 8:12].copy().view(np.uint32).reshape(n),
            "flags": raw[:, 12:16].copy().view(np.uint32).reshape(n),
            "copies": (raw[:, 12:16].copy().view(np.uint32).reshape(n) >> 8).astype(np.int64),
            "H2": raw[:, 16:20].copy().view(np.float32).reshape(n),
            "H3": raw[:, 20:24].copy().view(np.float32).reshape(n),
            "u0": raw[:, 24:28].copy().view(np.float32).reshape(n),
            "delta": raw[:, 28:32].copy().view(np.float32).reshape(n),
            "xhat": raw[:, 32:32 + 8 * K].copy().view(np.float32).reshape(n, 2 * K)}


def make_point(beta_p, E0, r, proposal=PROPOSAL_PAPER, point_id=0, logM=None, log_var_correction=None, sir_c=1.0):
    p = tkdv_point()
    p.beta_p, p.E0, p.r, p.proposal, p.point_id = beta_p, E0, r, proposal, point_id
    p.sir_c = float(sir_c)
    if logM is not None:
        p.override_logM, p.logM = 1, float(logM)
    if log_var_correction is not None:
        arr = np.ascontiguousarray(np.asarray(log_var_correction, dtype=np.float64))
        p._keep = arr  # keep alive until create copies it
        p.log_var_correction = arr.ctypes.data_as(C.POINTER(C.c_double))
    return p


def make_options(K, h3_mode=H3_TRIAD_F32, grid_N=0, sample_capacity=1 << 20, stream=None, use_graph=True,
                 ctas_per_sm=0, threads_per_cta=0, sir=False):
    """tkdv_options of a handle (include/tkdv.h)."""
    o = tkdv_options()
    o.K, o.h3_mode, o.grid_N = K, h3_mode, grid_N
    o.sample_capacity = sample_capacity
    if stream is None:
        o.cuda_stream = None  # the library makes its own stream
    else:
        handle = int(getattr(stream, "cuda_stream", stream))
        # handle 0 is the legacy default stream; pass cudaStreamLegacy (0x1) for it
        o.cuda_stream = C.c_void_p(handle if handle != 0 else 1)
    o.use_graph = 1 if use_graph else 0
    o.ctas_per_sm, o.threads_per_cta = ctas_per_sm, threads_per_cta
    o.sir = 1 if sir else 0
    return o


class Sampler:
    """One handle of the C library (several parameter points, one K)."""

    def __init__(self, K, points, h3_mode=H3_TRIAD_F32, grid_N=0, sample_capacity=1 << 20,
                 stream=None, use_graph=True, ctas_per_sm=0, threads_per_cta=0, sir=False):
        self.K = K
        self.n_points = len(points)
        o = make_options(K, h3_mode, grid_N, sample_capacity, stream, use_graph, ctas_per_sm, threads_per_cta, sir)
        self.h = sampler_create_ex(points, o)

    def run(self, n_proposals, seed):
        sampler_run(self.h, n_proposals, seed)

    def run_budgets(self, budgets, seed):
        sampler_run_budgets(self.h, budgets, seed)

    def run_ranges(self, idx0, count, seed):
        sampler_run_ranges(self.h, idx0, count, seed)

    def stats(self):
        return sampler_stats(self.h, self.n_points)

    def samples(self, max_records=1 << 20, device_dst=None, host_dst=None):
        return sampler_samples(self.h, self.K, max_records, device_dst, host_dst)

    def reset(self):
        sampler_reset(self.h)

    def sync(self):
        sampler_sync(self.h)

    def set_trace(self, dev_tensor, n):
        sampler_set_trace(self.h, dev_tensor, n)

    def set_deadline_ns(self, ns):
        sampler_set_deadline_ns(self.h, ns)

    def point_info(self, p=0):
        return sampler_point_info(self.h, p, self.K)

    def field_maxima(self, max_records=1 << 20):
        """Largest displacement (and its grid index j, xi_j = -pi + pi j/K) of
        each kept record, in the order samples() returns them."""
        return sampler_field_maxima(self.h, max_records)

    def extreme_field(self, m=500, point=0, max_records=1 << 20):
        """The 1-in-m event of Figs. 8-11: among the first m accepted fields
        of `point` (by proposal index) the one with the largest displacement
        on the 2K-point grid.  Returns a dict (idx, umax, xi, xhat) or None
        when fewer than m fields were kept."""
        rec = self.samples(max_records)
        umax, jm = self.field_maxima(max_records)
        sel = np.nonzero(rec["point"] == point)[0]
        if len(sel) < m:
            return None
        sel = sel[np.argsort(rec["idx"][sel], kind="stable")[:m]]
        b = sel[int(np.argmax(umax[sel]))]
        return {"idx": int(rec["idx"][b]), "umax": float(umax[b]),
                "xi": float(-np.pi + np.pi * jm[b] / self.K), "xhat": rec["xhat"][b].astype(np.float64)}

    def replay(self, p, idx, seed):
        return sampler_replay(self.h, p, self.K, idx, seed)

    def autotune(self, calib_proposals=1 << 22):
        return sampler_autotune(self.h, calib_proposals)

    def launch_config(self):
        return sampler_launch_config(self.h)

    def h3_form(self):
        return sampler_h3_form(self.h)

    def set_launch(self, variant, ctas_per_sm=0):
        sampler_set_launch(self.h, variant, ctas_per_sm)

    def close(self):
        if self.h:
            sampler_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
