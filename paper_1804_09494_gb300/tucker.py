"""Thin Python binding of libtucker (include/tucker.h).

Argument marshalling only: every step of the hot path runs in the CUDA
library; this module checks tensor placement, dtypes and shapes, passes raw
device pointers and torch's current CUDA stream, and turns status codes into
exceptions.  There is no CPU fallback: without the built library or a CUDA
device every call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtucker.so")

TUCKER_FP32 = 0
TUCKER_FP64 = 1
TUCKER_BF16X3 = 2
# context precision names: FP32 values with the Gram in split TF32 ("fp32" =
# "tf32x3") or split BF16 ("bf16x3"), or plain FP64
PREC = {"fp32": TUCKER_FP32, "tf32x3": TUCKER_FP32, "bf16x3": TUCKER_BF16X3, "fp64": TUCKER_FP64}
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_NUMERIC", 5: "ERR_TIMEOUT",
          6: "ERR_STATE", 7: "ERR_INDEX"}
PHASES = ("ttm_chain", "fixup", "gram", "eig", "backproj_cholqr2", "core_fit", "adjoint", "other")

# name -> (restype, argtypes); mirrors include/tucker.h
_VP = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_P64 = ctypes.POINTER(ctypes.c_int64)
_PD = ctypes.POINTER(ctypes.c_double)


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class Opts(ctypes.Structure):
    _fields_ = [("prec", _I32), ("P_bins", _I32), ("gauss_seidel", _I32), ("timing", _I32),
                ("wait_cap", _I32), ("ttm_path", _I32), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_user", _VP), ("svd", _I32), ("reserved", _I32 * 3)]


def torch_allocator(device):
    """(alloc, free) callbacks that hand the library memory from torch's
    caching allocator on `device` (marshalling only: the library decides what
    to allocate).  alloc returns NULL when torch cannot allocate."""
    dev = torch.device(device)

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
        except Exception:  # an exception must not cross the C boundary
            return None

    def _free(ptr, nbytes, stream, user):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    return ALLOC_FN(_alloc), FREE_FN(_free)


SIGNATURES = {
    "tucker_default_opts": (None, [ctypes.POINTER(Opts)]),
    "tucker_init": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, _P64, ctypes.POINTER(_I32), _I64,
                                   ctypes.POINTER(_VP), _VP, ctypes.POINTER(Opts), _VP]),
    "tucker_destroy": (None, [_VP]),
    "tucker_last_error": (ctypes.c_char_p, [_VP]),
    "tucker_stats": (ctypes.c_int, [_VP, ctypes.c_int, _P64, _P64, _P64, _P64, _P64]),
    "tucker_ttm_form": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), _P64]),
    "tucker_scheme_metrics": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _P64, _P64, _P64,
                                             _VP, _VP, _VP]),
    "tucker_partition": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP]),
    "tucker_partition_noalloc": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP]),
    "ttm_chain": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(_VP), _VP, _VP, _VP, _VP]),
    "factor_update": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, _VP]),
    "core": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), _VP, _VP]),
    "hooi_iter": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), _VP, _PD, _VP]),
    "ttm_chain_backward": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(_VP), _VP, _VP,
                                          ctypes.POINTER(_VP), _VP, _VP]),
    "tucker_timings": (ctypes.c_int, [_VP, _PD, _P64, ctypes.c_int, _VP]),
    "tucker_memory": (ctypes.c_int, [_VP, _P64]),
}

_lib = None


def load_library(path=LIB_PATH):
    """Loads libtucker.so and declares every entry point (no device work)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class TuckerError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _ptrs(ts):
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = t.data_ptr() if t is not None else 0
    return arr


def _need_cuda(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Tucker:
    """One COO tensor prepared for the HOOI hot path (wraps a tucker_t).

    idx  : (N, nnz) int32 CUDA tensor of 0-based coordinates (distinct)
    vals : (nnz,) float32 (prec "fp32", "tf32x3" or "bf16x3") or float64 (prec="fp64") CUDA tensor
    L, K : mode lengths and core lengths
    ttm_path : "auto" (the tensor-core TTM-chain where it applies), "cuda_cores", or "fiber"
               (CUDA cores, fiber-factored where the fiber mode is the second remaining mode)
    svd : "exact" (leading subspace of Z through its Gram matrix) or "lanczos"
          (the paper's Lanczos bidiagonalisation with 2K steps)
    """

    def __init__(self, idx, vals, L, K, prec="fp32", P_bins=0, gauss_seidel=False, timing=False,
                 wait_cap=0, allocator="torch", ttm_path="auto", svd="exact"):
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("libtucker needs a CUDA device")
        self.N = len(L)
        self.L = tuple(int(x) for x in L)
        self.K = tuple(int(x) for x in K)
        if prec not in PREC:
            raise ValueError(f"prec must be one of {sorted(PREC)}")
        self.prec = prec
        self.dtype = torch.float64 if prec == "fp64" else torch.float32
        _need_cuda(idx, torch.int32, "idx")
        _need_cuda(vals, self.dtype, "vals")
        if idx.dim() != 2 or idx.shape[0] != self.N or vals.shape != (idx.shape[1],):
            raise ValueError("idx must be (N, nnz) and vals (nnz,)")
        self.nnz = int(vals.shape[0])
        opts = Opts()
        self.lib.tucker_default_opts(ctypes.byref(opts))
        opts.prec = PREC[prec]
        opts.P_bins = int(P_bins)
        opts.gauss_seidel = int(bool(gauss_seidel))
        opts.timing = int(bool(timing))
        opts.wait_cap = int(wait_cap)
        paths = {"auto": 0, "cuda_cores": 1, "fiber": 2}
        if ttm_path not in paths:
            raise ValueError('ttm_path must be "auto", "cuda_cores" or "fiber"')
        opts.ttm_path = paths[ttm_path]
        if svd not in ("exact", "lanczos"):
            raise ValueError('svd must be "exact" or "lanczos"')
        opts.svd = 0 if svd == "exact" else 1
        # device memory from torch's caching allocator (allocator="torch"), or
        # the library's own cudaMalloc (allocator=None); the callbacks live as
        # long as the context
        self._allocator = torch_allocator(idx.device) if allocator == "torch" else None
        if self._allocator is not None:
            opts.alloc, opts.free = self._allocator
        Ls = (ctypes.c_int64 * self.N)(*self.L)
        Ks = (ctypes.c_int32 * self.N)(*self.K)
        rows = [idx[m] for m in range(self.N)]
        handle = ctypes.c_void_p()
        st = self.lib.tucker_init(ctypes.byref(handle), self.N, Ls, Ks, self.nnz, _ptrs(rows), _ptr(vals),
                                  ctypes.byref(opts), _stream())
        if st != 0:
            raise TuckerError(st, self.lib.tucker_last_error(None).decode())
        self.h = handle
        self.R = [self.stats(n)["R_n"] for n in range(self.N)]

    # ------------------------------------------------------------ plumbing
    def _check(self, st):
        if st != 0:
            raise TuckerError(st, self.lib.tucker_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.tucker_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def khat(self, n):
        out = 1
        for m in range(self.N):
            if m != n:
                out *= self.K[m]
        return out

    def _factors(self, F, skip=None):
        if len(F) != self.N:
            raise ValueError("need one factor per mode")
        for m, f in enumerate(F):
            if m == skip and f is None:
                continue
            _need_cuda(f, self.dtype, f"F[{m}]")
            if tuple(f.shape) != (self.L[m], self.K[m]):
                raise ValueError(f"F[{m}] must be {self.L[m]}x{self.K[m]}")
        return _ptrs(F)

    # ------------------------------------------------------------ entry points
    def stats(self, mode):
        v = [ctypes.c_int64() for _ in range(5)]
        self._check(self.lib.tucker_stats(self.h, mode, *[ctypes.byref(x) for x in v]))
        return dict(zip(("E_max", "R_sum", "R_max", "R_n", "P"), (x.value for x in v)))

    def scheme_metrics(self, mode, scheme, P, pos):
        """Section 4.1 metrics of CoarseG (scheme "coarseg") or MediumG ("mediumg")
        along `mode` for P processors; pos: N int32 CUDA tensors, pos[m][l] =
        position of index l of mode m in the random order.  Returns E_max,
        R_sum, R_max and the per-processor E, R (int64 CUDA tensors)."""
        code = {"coarseg": 1, "mediumg": 2}[scheme]
        for p in pos:
            _need_cuda(p, torch.int32, "pos")
        ptrs = (ctypes.c_void_p * self.N)(*[p.data_ptr() for p in pos])
        E = torch.empty(P, dtype=torch.int64, device="cuda")
        R = torch.empty(P, dtype=torch.int64, device="cuda")
        v = [ctypes.c_int64() for _ in range(3)]
        self._check(self.lib.tucker_scheme_metrics(self.h, mode, code, int(P), ptrs, *[ctypes.byref(x) for x in v],
                                                   _ptr(E), _ptr(R), _stream()))
        return dict(E_max=v[0].value, R_sum=v[1].value, R_max=v[2].value, E=E, R=R)

    def ttm_form(self, mode):
        """{"tensor_cores": bool, "blocks": padded 8-element blocks (0 on CUDA cores)}"""
        tc, nb = ctypes.c_int32(), ctypes.c_int64()
        self._check(self.lib.tucker_ttm_form(self.h, mode, ctypes.byref(tc), ctypes.byref(nb)))
        return {"tensor_cores": bool(tc.value), "blocks": nb.value}

    def partition(self, mode):
        P = self.stats(mode)["P"]
        bin_ptr = torch.empty(P + 1, dtype=torch.int64, device="cuda")
        perm = torch.empty(self.nnz, dtype=torch.int32, device="cuda")
        self._check(self.lib.tucker_partition(self.h, mode, _ptr(bin_ptr), _ptr(perm), _stream()))
        return bin_ptr, perm

    def partition_noalloc(self, mode, bin_ptr, perm):
        """tucker_partition_noalloc into caller-owned outputs (P+1 int64, nnz int32)."""
        _need_cuda(bin_ptr, torch.int64, "bin_ptr")
        _need_cuda(perm, torch.int32, "perm")
        self._check(self.lib.tucker_partition_noalloc(self.h, mode, _ptr(bin_ptr), _ptr(perm), _stream()))
        return bin_ptr, perm

    def ttm_chain(self, mode, F, vals=None, out=None, row_id=True):
        Fp = self._factors(F, skip=mode)
        if vals is not None:
            _need_cuda(vals, self.dtype, "vals")
        Z = out if out is not None else torch.empty(self.R[mode], self.khat(mode), dtype=self.dtype, device="cuda")
        _need_cuda(Z, self.dtype, "Z")
        rid = torch.empty(self.R[mode], dtype=torch.int32, device="cuda") if row_id else None
        self._check(self.lib.ttm_chain(self.h, mode, Fp, _ptr(vals), _ptr(Z), _ptr(rid), _stream()))
        return Z, rid

    def factor_update(self, mode, Z, out=None):
        _need_cuda(Z, self.dtype, "Z")
        F = out if out is not None else torch.empty(self.L[mode], self.K[mode], dtype=self.dtype, device="cuda")
        sigma = torch.empty(self.K[mode], dtype=torch.float64, device="cuda")
        self._check(self.lib.factor_update(self.h, mode, _ptr(Z), _ptr(F), _ptr(sigma), _stream()))
        return F, sigma

    def core(self, F, out=None):
        Fp = self._factors(F)
        size = 1
        for k in self.K:
            size *= k
        G = out if out is not None else torch.empty(size, dtype=self.dtype, device="cuda")
        self._check(self.lib.core(self.h, Fp, _ptr(G), _stream()))
        return G

    def hooi_iter(self, F, G=None, want_fit=True):
        """One HOOI invocation; updates the tensors in F in place."""
        Fp = self._factors(F)
        size = 1
        for k in self.K:
            size *= k
        G = G if G is not None else torch.empty(size, dtype=self.dtype, device="cuda")
        fit = ctypes.c_double(float("nan"))
        self._check(self.lib.hooi_iter(self.h, Fp, _ptr(G), ctypes.byref(fit) if want_fit else None, _stream()))
        return G, (fit.value if want_fit else None)

    def ttm_chain_backward(self, mode, F, dZ, vals=None, dF=None, want_dval=True):
        Fp = self._factors(F, skip=mode)
        _need_cuda(dZ, self.dtype, "dZ")
        if vals is not None:
            _need_cuda(vals, self.dtype, "vals")
        if dF is None:
            dF = [None if m == mode else torch.zeros(self.L[m], self.K[m], dtype=self.dtype, device="cuda")
                  for m in range(self.N)]
        dval = torch.empty(self.nnz, dtype=self.dtype, device="cuda") if want_dval else None
        self._check(self.lib.ttm_chain_backward(self.h, mode, Fp, _ptr(dZ), _ptr(vals), _ptrs(dF), _ptr(dval),
                                                _stream()))
        return dF, dval

    def timings(self, reset=False):
        ms = (ctypes.c_double * 8)()
        ln = (ctypes.c_int64 * 8)()
        self._check(self.lib.tucker_timings(self.h, ms, ln, int(reset), _stream()))
        return {p: (ms[i], ln[i]) for i, p in enumerate(PHASES)}

    def memory(self):
        b = ctypes.c_int64()
        self._check(self.lib.tucker_memory(self.h, ctypes.byref(b)))
        return b.value


class TTMChain(torch.autograd.Function):
    """Z = ttm_chain(vals, F) with the hand-written adjoint as its backward:
    dvals(e) = <dZ[row(e)], Kron_n(e)>, dF_m from ttm_chain_backward."""

    @staticmethod
    def forward(ctx, tk, mode, vals, *F):
        ctx.tk, ctx.mode = tk, mode
        ctx.save_for_backward(vals, *F)
        Z, _ = tk.ttm_chain(mode, list(F), vals=vals, row_id=False)
        return Z

    @staticmethod
    def backward(ctx, dZ):
        vals, *F = ctx.saved_tensors
        dF, dval = ctx.tk.ttm_chain_backward(ctx.mode, F, dZ.contiguous(), vals=vals)
        return (None, None, dval) + tuple(dF)


class KronGather(torch.autograd.Function):
    """x(e) = <W[row(l_n(e))], Kron_n(e)> for every element (the adjoint of the
    TTM-chain in the values).  Backward: dW = ttm_chain(vals=g), dF_m from the
    adjoint with weights g."""

    @staticmethod
    def forward(ctx, tk, mode, W, *F):
        ctx.tk, ctx.mode = tk, mode
        ctx.save_for_backward(W, *F)
        _, x = tk.ttm_chain_backward(mode, list(F), W.contiguous(), dF=[None] * tk.N)
        return x

    @staticmethod
    def backward(ctx, g):
        W, *F = ctx.saved_tensors
        g = g.contiguous()
        dW, _ = ctx.tk.ttm_chain(ctx.mode, F, vals=g, row_id=False)
        dF, _ = ctx.tk.ttm_chain_backward(ctx.mode, F, W.contiguous(), vals=g, want_dval=False)
        return (None, None, dW) + tuple(dF)
