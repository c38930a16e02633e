"""Thin ctypes binding over libplnmf.so (include/nmf.h).

Argument marshalling only: every step of the factorisation runs in the CUDA
library.  Arrays may be torch tensors (device or host) or numpy arrays (host);
the binding passes their data pointers.  Importing this module loads the
library and raises if it has not been built.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libplnmf.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -m paper_1904_07935_b300.build` "
        "(there is no CPU fallback)")

lib = ctypes.CDLL(LIB_PATH)

NMF_OK, NMF_EINVAL, NMF_ENOMEM, NMF_ECUDA, NMF_ETIMEOUT, NMF_ENUMERIC, NMF_EBUSY, NMF_EUNSUPPORTED = range(8)
DENSE_F32, CSR_F32_I32 = 0, 1
PREC_FP32, PREC_BF16 = 0, 1
STEP_R, STEP_S, STEP_UPDATE_H, STEP_P, STEP_Q, STEP_UPDATE_W, STEP_OBJECTIVE = range(7)
BUF_W, BUF_HT, BUF_R, BUF_P, BUF_S, BUF_Q = range(6)


class Problem(ctypes.Structure):
    _fields_ = [
        ("V", ctypes.c_int32), ("D", ctypes.c_int32), ("K", ctypes.c_int32),
        ("fmt", ctypes.c_int32),
        ("dense", ctypes.c_void_p), ("ld", ctypes.c_int64),
        ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p),
        ("nnz", ctypes.c_int64),
        ("W0", ctypes.c_void_p), ("H0", ctypes.c_void_p),
        ("seed", ctypes.c_uint64), ("eps", ctypes.c_float), ("tile_T", ctypes.c_int32),
        ("prec", ctypes.c_int32), ("stream", ctypes.c_void_p), ("flags", ctypes.c_int32),
    ]


FLAG_TC_GRAMS = 1
FLAG_MULTI_LAUNCH_W = 2
FLAG_NO_TMA = 4
FLAG_BF16_SINGLE_A = 8
FLAG_BF16_SINGLE_FACTORS = 16
FLAG_TC_UPDATES = 32


_vp, _i32, _i64, _dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "nmf_init": ([ctypes.POINTER(Problem), ctypes.POINTER(_vp)], _i32),
    "nmf_iterate": ([_vp, _i32], _i32),
    "nmf_error": ([_vp, _dp, _dp], _i32),
    "nmf_objective_history": ([_vp, _vp, _i32], _i32),
    "nmf_get_factors": ([_vp, _vp, _vp], _i32),
    "nmf_set_factors": ([_vp, _vp, _vp], _i32),
    "nmf_iterate_host": ([_vp, _vp, _vp, _vp, _vp, _dp], _i32),
    "nmf_run_step": ([_vp, _i32], _i32),
    "nmf_get_buffer": ([_vp, _i32, _vp, _i64], _i32),
    "nmf_set_buffer": ([_vp, _i32, _vp, _i64], _i32),
    "nmf_query": ([_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)], _i32),
    "nmf_set_wait_limits": ([_vp, _i64, _i32], _i32),
    "nmf_set_w_workers_after_chain": ([_vp, _i32], _i32),
    "nmf_set_spmm_split": ([_vp, _i32, _i32], _i32),
    "nmf_tune_spmm": ([_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)], _i32),
    "nmf_query_form": ([_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)], _i32),
    "nmf_profile": ([_vp, _i32, _vp], _i32),
    "nmf_iterate_alg1": ([_vp, _i32, _vp], _i32),
    "nmf_iterate_mu": ([_vp, _i32, _vp], _i32),
    "nmf_destroy": ([_vp], None),
    "nmf_gram_noalloc": ([_vp, _i32, _i32, _i64, _vp, _vp], _i32),
    "nmf_gemm": ([_i32, _i32, _i32, _vp, _i64, _i32, _vp, _i64, _vp, _i64, _i32, _vp], _i32),
    "nmf_gemm_bf16": ([_i32, _i32, _i32, _vp, _i64, _vp, _i64, _vp, _i64, _vp], _i32),
    "nmf_batch_create": ([_vp, _i32, _i32, _vp, _vp], _i32),
    "nmf_batch_iterate": ([_vp, _i32], _i32),
    "nmf_batch_query": ([_vp, _i32, _vp, _vp], _i32),
    "nmf_batch_query_schedule": ([_vp, _i32, _vp, _vp, _vp], _i32),
    "nmf_batch_destroy": ([_vp], None),
    "nmf_batch_submit": ([_vp, _i32, _i32, _vp], _i32),
    "nmf_mlp_create": ([_i32, _i32, ctypes.c_uint64, _vp], _i32),
    "nmf_mlp_set_params": ([_vp, _vp], _i32),
    "nmf_mlp_get_params": ([_vp, _vp], _i32),
    "nmf_mlp_forward": ([_vp, _vp, _i32, _vp, _vp], _i32),
    "nmf_mlp_grads": ([_vp, _vp, _vp, _i32, _vp, _vp], _i32),
    "nmf_mlp_train_step": ([_vp, _vp, _vp, _i32, ctypes.c_float, _vp, _vp], _i32),
    "nmf_mlp_destroy": ([_vp], None),
    "nmf_warm_h": ([_vp, _vp, _vp, ctypes.c_float, _i32, _vp, _vp, _vp, _vp, _vp], _i32),
    "nmf_status_str": ([_i32], ctypes.c_char_p),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res


class NmfError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {lib.nmf_status_str(status).decode()} (status {status})")


def check(status: int, where: str) -> None:
    if status != NMF_OK:
        raise NmfError(status, where)


def ptr(x) -> int | None:
    """Data pointer of a torch tensor / numpy array (must be contiguous)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(type(x))


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def problem_struct(V, D, K, *, dense=None, ld=None, row_ptr=None, col_idx=None, val=None, W0=None, H0=None,
                   seed=0, eps=0.0, tile_T=0, prec=PREC_FP32, stream=None, flags=0):
    """nmf_problem for device tensors; returns (struct, objects to keep alive)."""
    p = Problem()
    p.V, p.D, p.K = V, D, K
    keep = [dense, row_ptr, col_idx, val, W0, H0]
    if dense is not None:
        p.fmt = DENSE_F32
        p.dense = ptr(dense)
        p.ld = D if ld is None else ld
    else:
        p.fmt = CSR_F32_I32
        p.row_ptr, p.col_idx, p.val = ptr(row_ptr), ptr(col_idx), ptr(val)
        p.nnz = int(val.shape[0]) if val is not None else 0
    p.W0, p.H0 = ptr(W0), ptr(H0)
    p.seed, p.eps, p.tile_T, p.prec = seed, eps, tile_T, prec
    p.stream = _stream_ptr(stream)
    p.flags = flags
    return p, keep


class Nmf:
    """One factorisation context (nmf_ctx)."""

    def __init__(self, V, D, K, *, dense=None, ld=None, row_ptr=None, col_idx=None, val=None,
                 W0=None, H0=None, seed=0, eps=0.0, tile_T=0, prec=PREC_FP32, stream=None, flags=0, _handle=None):
        if _handle is not None:                      # adopt a context made by nmf_batch_submit
            self.h, self._keep = _handle, []
            self.V, self.D, self.K = V, D, K
            return
        p, self._keep = problem_struct(V, D, K, dense=dense, ld=ld, row_ptr=row_ptr, col_idx=col_idx, val=val,
                                       W0=W0, H0=H0, seed=seed, eps=eps, tile_T=tile_T, prec=prec,
                                       stream=stream, flags=flags)
        h = ctypes.c_void_p()
        check(lib.nmf_init(ctypes.byref(p), ctypes.byref(h)), "nmf_init")
        self.h = h
        self.V, self.D, self.K = V, D, K

    # context management
    def close(self):
        if getattr(self, "h", None):
            lib.nmf_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # calls
    def iterate(self, n=1):
        check(lib.nmf_iterate(self.h, n), "nmf_iterate")

    def error(self):
        f, r = ctypes.c_double(), ctypes.c_double()
        check(lib.nmf_error(self.h, ctypes.byref(f), ctypes.byref(r)), "nmf_error")
        return f.value, r.value

    def history(self, n):
        out = np.empty(n, dtype=np.float64)
        check(lib.nmf_objective_history(self.h, out.ctypes.data, n), "nmf_objective_history")
        return out

    def get_factors(self, W=None, H=None):
        """Returns host numpy (W V x K, H K x D) unless destinations are given."""
        ret = W is None and H is None
        if ret:
            W = np.empty((self.V, self.K), dtype=np.float32)
            H = np.empty((self.K, self.D), dtype=np.float32)
        check(lib.nmf_get_factors(self.h, ptr(W), ptr(H)), "nmf_get_factors")
        return (W, H) if ret else None

    def set_factors(self, W=None, H=None):
        check(lib.nmf_set_factors(self.h, ptr(W), ptr(H)), "nmf_set_factors")

    def iterate_host(self, W_in=None, H_in=None, W_out=None, H_out=None):
        """One iteration on caller-held factors (W V x K, H K x D; pinned
        host or device buffers overlap the copies with the iteration); the
        outputs may be the inputs.  Returns the objective after it."""
        f = ctypes.c_double()
        check(lib.nmf_iterate_host(self.h, ptr(W_in), ptr(H_in), ptr(W_out), ptr(H_out), ctypes.byref(f)),
              "nmf_iterate_host")
        return f.value

    def run_step(self, step):
        check(lib.nmf_run_step(self.h, step), "nmf_run_step")

    _SHAPES = {BUF_W: ("V", "K"), BUF_HT: ("D", "K"), BUF_R: ("D", "K"), BUF_P: ("V", "K"),
               BUF_S: ("K", "K"), BUF_Q: ("K", "K")}

    def buffer_shape(self, which):
        a, b = self._SHAPES[which]
        return getattr(self, a), getattr(self, b)

    def get_buffer(self, which, out=None):
        shape = self.buffer_shape(which)
        if out is None:
            out = np.empty(shape, dtype=np.float32)
        check(lib.nmf_get_buffer(self.h, which, ptr(out), shape[0] * shape[1]), "nmf_get_buffer")
        return out

    def set_buffer(self, which, src):
        shape = self.buffer_shape(which)
        if isinstance(src, np.ndarray):
            src = np.ascontiguousarray(src, dtype=np.float32)
        check(lib.nmf_set_buffer(self.h, which, ptr(src), shape[0] * shape[1]), "nmf_set_buffer")

    PROFILE_STEPS = ("R", "update_H", "P", "Q", "update_W", "S", "objective")

    def profile(self, n_iters):
        """Mean ms per iteration of each step (eager launches, CUDA events)."""
        out = np.zeros(len(self.PROFILE_STEPS), dtype=np.float32)
        check(lib.nmf_profile(self.h, n_iters, out.ctypes.data), "nmf_profile")
        return dict(zip(self.PROFILE_STEPS, out.tolist()))

    def iterate_alg1(self, n=1, profile=False):
        """n iterations of Alg. 1 as written (column by column, no tiling);
        with profile=True the mean ms of each step (as profile())."""
        if profile:
            out = np.zeros(len(self.PROFILE_STEPS), dtype=np.float32)
            check(lib.nmf_iterate_alg1(self.h, n, out.ctypes.data), "nmf_iterate_alg1")
            return dict(zip(self.PROFILE_STEPS, out.tolist()))
        check(lib.nmf_iterate_alg1(self.h, n, None), "nmf_iterate_alg1")

    def iterate_mu(self, n=1, profile=False):
        """n multiplicative-update iterations (Lee & Seung); with profile=True
        the mean ms of each step (as profile())."""
        if profile:
            out = np.zeros(len(self.PROFILE_STEPS), dtype=np.float32)
            check(lib.nmf_iterate_mu(self.h, n, out.ctypes.data), "nmf_iterate_mu")
            return dict(zip(self.PROFILE_STEPS, out.tolist()))
        check(lib.nmf_iterate_mu(self.h, n, None), "nmf_iterate_mu")

    def query(self):
        t, c, l = _i32(), _i32(), _i32()
        check(lib.nmf_query(self.h, ctypes.byref(t), ctypes.byref(c), ctypes.byref(l)), "nmf_query")
        w1, sw, sn = _i32(), _i32(), _i32()
        check(lib.nmf_query_form(self.h, ctypes.byref(w1), ctypes.byref(sw), ctypes.byref(sn)), "nmf_query_form")
        return {"tile_T": t.value, "chain_ctas": c.value, "launches_per_iter": l.value,
                "w_single_launch": bool(w1.value), "s_in_w_update": bool(sw.value), "s_chunks": sn.value}

    def set_wait_limits(self, wait_ns=0, extra_arrivals=0):
        """Limit of the W update's device waits (0: library default) and, for
        tests of the failure path, extra chain arrivals the base-forming CTAs
        wait for (include/nmf.h, nmf_set_wait_limits)."""
        check(lib.nmf_set_wait_limits(self.h, int(wait_ns), int(extra_arrivals)), "nmf_set_wait_limits")

    def set_spmm_split(self, seg_P, seg_R):
        """Split lengths of the sparse products' long rows (0: no split;
        include/nmf.h, nmf_set_spmm_split)."""
        check(lib.nmf_set_spmm_split(self.h, int(seg_P), int(seg_R)), "nmf_set_spmm_split")

    def tune_spmm(self):
        """Time the sparse products' split lengths and keep the fastest;
        returns (seg_P, seg_R), 0 meaning no split (nmf_tune_spmm)."""
        sp, sr = _i32(0), _i32(0)
        check(lib.nmf_tune_spmm(self.h, ctypes.byref(sp), ctypes.byref(sr)), "nmf_tune_spmm")
        return sp.value, sr.value

    def set_w_workers_after_chain(self, on=True):
        """Run the W update's worker grid after its chain grid instead of
        beside it (include/nmf.h, nmf_set_w_workers_after_chain)."""
        check(lib.nmf_set_w_workers_after_chain(self.h, 1 if on else 0), "nmf_set_w_workers_after_chain")


def gemm(A, B, C, *, transA=False, prec=PREC_FP32, stream=None):
    """C = op(A) @ B on the tensor cores (device tensors, row-major)."""
    M, N = C.shape
    K = A.shape[0] if transA else A.shape[1]
    check(lib.nmf_gemm(M, N, K, ptr(A), A.shape[1], 1 if transA else 0, ptr(B), B.shape[1], ptr(C), C.shape[1],
                       prec, _stream_ptr(stream)), "nmf_gemm")


class Batch:
    """Contexts advanced together by one CUDA graph (nmf_batch)."""

    def __init__(self, members, *, autotune=True, stream=None):
        arr = (ctypes.c_void_p * len(members))(*[m.h.value for m in members])
        h = ctypes.c_void_p()
        check(lib.nmf_batch_create(arr, len(members), 1 if autotune else 0, _stream_ptr(stream), ctypes.byref(h)),
              "nmf_batch_create")
        self.h = h
        self.members = list(members)

    def iterate(self, n=1):
        check(lib.nmf_batch_iterate(self.h, n), "nmf_batch_iterate")

    def query(self, i):
        """(chain cluster size, autotuned W-update microseconds) of member i."""
        cl, us = ctypes.c_int32(), ctypes.c_float()
        check(lib.nmf_batch_query(self.h, i, ctypes.byref(cl), ctypes.byref(us)), "nmf_batch_query")
        return cl.value, us.value

    def schedule(self, i):
        """Member i's autotuned W tile width and SpMM split lengths (P, R)."""
        t, sp, sr = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(lib.nmf_batch_query_schedule(self.h, i, ctypes.byref(t), ctypes.byref(sp), ctypes.byref(sr)),
              "nmf_batch_query_schedule")
        return {"tile_T": t.value, "spmm_seg_P": sp.value, "spmm_seg_R": sr.value}

    def close(self):
        if getattr(self, "h", None):
            lib.nmf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def sparse_device(prob, device="cuda"):
    """CSR arrays of a synth.SparseProblem on the device (torch tensors)."""
    import torch
    A = prob.A
    return (torch.from_numpy(A.row_ptr).to(device), torch.from_numpy(A.col_idx).to(device),
            torch.from_numpy(A.val).to(device))


def batch_submit(specs, n_iters):
    """nmf_batch_submit.  specs: list of dicts of problem_struct keyword
    arguments (V, D, K and the device arrays).  Returns Nmf objects owning the
    contexts."""
    structs, keep = [], []
    for s in specs:
        p, k = problem_struct(**s)
        structs.append(p)
        keep.append(k)
    arr = (Problem * len(structs))(*structs)
    outs = (ctypes.c_void_p * len(structs))()
    check(lib.nmf_batch_submit(arr, len(structs), n_iters, outs), "nmf_batch_submit")
    res = []
    for s, k, h in zip(specs, keep, outs):
        m = Nmf(s["V"], s["D"], s["K"], _handle=ctypes.c_void_p(h))
        m._keep = k
        res.append(m)
    return res


class Mlp:
    """Warm-start network K -> hidden -> hidden -> K (nmf_mlp)."""

    def __init__(self, K, hidden=256, seed=0):
        h = ctypes.c_void_p()
        check(lib.nmf_mlp_create(K, hidden, seed, ctypes.byref(h)), "nmf_mlp_create")
        self.h, self.K, self.hidden = h, K, hidden

    def shapes(self):
        K, H = self.K, self.hidden
        return [(K, H), (H,), (H, H), (H,), (H, K), (K,)]

    def set_params(self, params):
        arrs = [np.ascontiguousarray(p, dtype=np.float32) for p in params]
        for a, s in zip(arrs, self.shapes()):
            if a.shape != s:
                raise ValueError(f"parameter shape {a.shape} != {s}")
        ptrs = (ctypes.c_void_p * 6)(*[a.ctypes.data for a in arrs])
        check(lib.nmf_mlp_set_params(self.h, ptrs), "nmf_mlp_set_params")

    def get_params(self):
        arrs = [np.empty(s, dtype=np.float32) for s in self.shapes()]
        ptrs = (ctypes.c_void_p * 6)(*[a.ctypes.data for a in arrs])
        check(lib.nmf_mlp_get_params(self.h, ptrs), "nmf_mlp_get_params")
        return arrs

    def forward(self, X, Y=None, stream=None):
        """X: rows x K float32 CUDA tensor; returns Y (CUDA tensor)."""
        import torch
        if Y is None:
            Y = torch.empty_like(X)
        check(lib.nmf_mlp_forward(self.h, ptr(X), X.shape[0], ptr(Y), _stream_ptr(stream)), "nmf_mlp_forward")
        return Y

    def grads(self, X, T):
        arrs = [np.empty(s, dtype=np.float32) for s in self.shapes()]
        ptrs = (ctypes.c_void_p * 6)(*[a.ctypes.data for a in arrs])
        loss = ctypes.c_double()
        check(lib.nmf_mlp_grads(self.h, ptr(X), ptr(T), X.shape[0], ptrs, ctypes.byref(loss)), "nmf_mlp_grads")
        return arrs, loss.value

    def train_step(self, X, T, lr=1e-3, want_loss=False, stream=None):
        loss = ctypes.c_double()
        check(lib.nmf_mlp_train_step(self.h, ptr(X), ptr(T), X.shape[0], lr,
                                     ctypes.byref(loss) if want_loss else None, _stream_ptr(stream)),
              "nmf_mlp_train_step")
        return loss.value if want_loss else None

    def close(self):
        if getattr(self, "h", None):
            lib.nmf_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def warm_h(ctx, prob, *, mlp=None, tol=1e-3, max_sweeps=100, H_ref=None, want_R=False, seed=0):
    """nmf_warm_h for the new documents of a synth.SparseProblem (V x N CSR).
    Returns dict(H (K x N), R (N x K) or None, sweeps, trace)."""
    import torch
    A = prob.A
    rp, ci, va = sparse_device(prob)
    p, keep = problem_struct(A.n_rows, A.n_cols, ctx.K, row_ptr=rp, col_idx=ci, val=va, seed=seed)
    N, K = A.n_cols, ctx.K
    H = np.empty((K, N), dtype=np.float32)
    R = np.empty((N, K), dtype=np.float32) if want_R else None
    href = None
    if H_ref is not None:
        href = H_ref if hasattr(H_ref, "data_ptr") else np.ascontiguousarray(H_ref, dtype=np.float32)
    sweeps = ctypes.c_int32()
    trace = np.zeros(max(1, max_sweeps), dtype=np.float64)
    check(lib.nmf_warm_h(ctx.h, mlp.h if mlp is not None else None, ctypes.byref(p), tol, max_sweeps, ptr(href),
                         H.ctypes.data, ptr(R), ctypes.byref(sweeps), trace.ctypes.data), "nmf_warm_h")
    del keep
    return {"H": H, "R": R, "sweeps": sweeps.value, "trace": trace[:sweeps.value]}


def gemm_bf16(A, B, C, *, stream=None):
    """C = A @ B^T with A (M x K) and B (N x K) torch.bfloat16 device tensors
    (row strides multiples of 8), C float32 (M x N)."""
    M, N = C.shape
    K = A.shape[1]
    for x in (A, B, C):
        if x.stride(1) != 1:
            raise ValueError("rows must be contiguous")
    check(lib.nmf_gemm_bf16(M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), C.data_ptr(),
                            C.stride(0), _stream_ptr(stream)), "nmf_gemm_bf16")


def gram_noalloc(X, S, *, stream=None):
    """S = X^T X through nmf_gram_noalloc (device tensors, row-major)."""
    N, K = X.shape
    check(lib.nmf_gram_noalloc(ptr(X), N, K, X.stride(0), ptr(S), _stream_ptr(stream)), "nmf_gram_noalloc")


def from_sparse(prob, K, device="cuda", **kw):
    """Context for a synth.SparseProblem; copies its CSR to the device with torch."""
    import torch
    A = prob.A
    rp = torch.from_numpy(A.row_ptr).to(device)
    ci = torch.from_numpy(A.col_idx).to(device)
    va = torch.from_numpy(A.val).to(device)
    ctx = Nmf(A.n_rows, A.n_cols, K, row_ptr=rp, col_idx=ci, val=va, **kw)
    ctx._keep += [rp, ci, va]
    return ctx


def from_dense(A, K, device="cuda", **kw):
    """Context for a dense float32 matrix (numpy or torch)."""
    import torch
    if isinstance(A, np.ndarray):
        A = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32))
    A = A.to(device).contiguous()
    ctx = Nmf(A.shape[0], A.shape[1], K, dense=A, **kw)
    ctx._keep.append(A)
    return ctx
