"""Python binding of the C ABI (argument marshalling only).

Every step of the search runs in libtpuknn.so; torch provides device memory
and streams. See include/tpuknn.h for the semantics of each call.
"""
import torch

from . import _lib
from ._lib import METRIC, DTYPE, BINS, check

_ESIZE = {"f32": 4, "bf16": 2, "e4m3": 1, "e4m3t": 1}


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t):
    return None if t is None else t.data_ptr()


def plan_bins(N, K, recall_target=0.95, round_to=1):
    """Eq. 14: bins for an expected recall (Eq. 13) of at least recall_target."""
    L = _lib.get().knn_plan_bins(int(N), int(K), float(recall_target), int(round_to))
    if L < 1:
        raise ValueError("no bin count for N=%d K=%d r=%g" % (N, K, recall_target))
    return int(L)


def row_pitch(D):
    return int(_lib.get().knn_row_pitch(int(D)))


def _workspace(nbytes, device):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


class Database:
    """A device-resident database prepared for search (knn_prepare).

    x: N x D float32 CUDA tensor. metric: 'ip' | 'l2' | 'cos'.
    dtype: 'f32' | 'bf16' | 'e4m3' (per-row scales) | 'e4m3t' (one scale for
    the whole database) -- the contraction's element type.
    keep_f32: keep FP32 rows for the final re-rank (for 'cos' the
    unit-length copy is always kept; otherwise this holds a reference to x).
    """

    def __init__(self, x, metric="l2", dtype="bf16", keep_f32=True, stream=None):
        if not (x.is_cuda and x.dtype == torch.float32 and x.dim() == 2):
            raise ValueError("x must be a 2-D float32 CUDA tensor")
        x = x.contiguous()
        self.N, self.D = x.shape
        self.metric, self.dtype = metric, dtype
        self.device = x.device
        self.pitch = row_pitch(self.D)
        dev = x.device
        self.lp = torch.empty(self.N * self.pitch * _ESIZE[dtype], dtype=torch.uint8, device=dev)
        self.scale = (torch.empty(self.N, dtype=torch.float32, device=dev)
                      if dtype in ("e4m3", "e4m3t") else None)
        self.hnorm = torch.empty(self.N, dtype=torch.float32, device=dev) if metric == "l2" else None
        if metric == "cos":
            self.f32 = torch.empty((self.N, self.D), dtype=torch.float32, device=dev)
        else:
            self.f32 = x if keep_f32 else None
        with torch.cuda.device(dev):
            check(_lib.get().knn_prepare(x.data_ptr(), self.N, self.D, METRIC[metric], DTYPE[dtype],
                                         self.lp.data_ptr(), _ptr(self.scale), _ptr(self.hnorm),
                                         _ptr(self.f32) if metric == "cos" else None,
                                         _stream(stream)), "knn_prepare")
        self._ws = {}

    # -- helpers ---------------------------------------------------------------
    def _args(self):
        return (self.lp.data_ptr(), _ptr(self.scale), _ptr(self.hnorm), _ptr(self.f32),
                self.N, self.D, DTYPE[self.dtype], METRIC[self.metric])

    def _get_ws(self, key, nbytes):
        ws = self._ws.get(key)
        if ws is None or ws.numel() < nbytes:
            ws = _workspace(nbytes, self.device)
            self._ws[key] = ws
        return ws

    def resolve_L(self, K, L=None, recall_target=0.95):
        return int(L) if L else plan_bins(self.N, K, recall_target)

    # -- calls -----------------------------------------------------------------
    def search(self, q, K, L=None, recall_target=0.95, rerank=2, stream=None, out=None,
               bins="mod", slot=0):
        """Approximate search; returns (values M x K float32, indices M x K int32).

        bins: "mod" (row j in bin j mod L) or "contiguous" (runs of rows).
        slot: each slot has its own workspace; searches in flight on different
        streams at the same time use different slots."""
        q = q.contiguous()
        M = q.shape[0]
        L = self.resolve_L(K, L, recall_target)
        lib = _lib.get()
        nb = lib.knn_search_workspace(self.N, self.D, DTYPE[self.dtype], METRIC[self.metric], M, K,
                                      L, BINS[bins], recall_target, rerank)
        if nb == 0:
            raise ValueError("invalid search arguments (N=%d D=%d M=%d K=%d L=%d)"
                             % (self.N, self.D, M, K, L))
        ws = self._get_ws(("search", M, K, L, rerank, bins, slot), nb)
        if out is None:
            val = torch.empty((M, K), dtype=torch.float32, device=self.device)
            idx = torch.empty((M, K), dtype=torch.int32, device=self.device)
        else:
            val, idx = out
        with torch.cuda.device(self.device):
            check(lib.knn_search(*self._args(), q.data_ptr(), M, K, L, BINS[bins], recall_target,
                                 rerank, val.data_ptr(), idx.data_ptr(), ws.data_ptr(),
                                 ws.numel(), _stream(stream)), "knn_search")
        return val, idx

    def search_host(self, q_host, K, L=None, recall_target=0.95, rerank=2, stream=None,
                    out=None, bins="mod", wait=True, slot=0):
        """Search with host queries and host outputs (copies inside the call).

        wait=False enqueues the work on `stream` and returns at once
        (knn_search_host_async): the outputs are valid, and q_host and the
        outputs reusable, once the stream has completed it. Each `slot` has its
        own workspace, so calls in flight on different streams use different
        slots."""
        M = q_host.shape[0]
        L = self.resolve_L(K, L, recall_target)
        lib = _lib.get()
        nb = lib.knn_search_host_workspace(self.N, self.D, DTYPE[self.dtype], METRIC[self.metric],
                                           M, K, L, BINS[bins], recall_target, rerank)
        if nb == 0:
            raise ValueError("invalid search arguments")
        ws = self._get_ws(("host", M, K, L, rerank, bins, slot), nb)
        if out is None:
            val = torch.empty((M, K), dtype=torch.float32, pin_memory=True)
            idx = torch.empty((M, K), dtype=torch.int32, pin_memory=True)
        else:
            val, idx = out
        fn = lib.knn_search_host if wait else lib.knn_search_host_async
        with torch.cuda.device(self.device):
            check(fn(*self._args(), q_host.data_ptr(), M, K, L, BINS[bins], recall_target, rerank,
                     val.data_ptr(), idx.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)),
                  "knn_search_host" if wait else "knn_search_host_async")
        return val, idx

    def search_static(self, q, K, L=None, recall_target=0.95, rerank=2, stream=None, out=None,
                      bins="mod"):
        """search() in the library's own scratch buffer (knn_search_static): no
        workspace is allocated; out= preallocated outputs make the call
        allocation-free on the Python side too."""
        q = q.contiguous()
        M = q.shape[0]
        L = self.resolve_L(K, L, recall_target)
        if out is None:
            val = torch.empty((M, K), dtype=torch.float32, device=self.device)
            idx = torch.empty((M, K), dtype=torch.int32, device=self.device)
        else:
            val, idx = out
        with torch.cuda.device(self.device):
            check(_lib.get().knn_search_static(*self._args(), q.data_ptr(), M, K, L, BINS[bins],
                                               recall_target, rerank, val.data_ptr(),
                                               idx.data_ptr(), _stream(stream)),
                  "knn_search_static")
        return val, idx

    def search_exact(self, q, K, stream=None):
        q = q.contiguous()
        M = q.shape[0]
        lib = _lib.get()
        nb = lib.knn_search_exact_workspace(self.N, self.D, DTYPE[self.dtype], METRIC[self.metric],
                                            M, K)
        if nb == 0:
            raise ValueError("invalid exact-search arguments")
        ws = self._get_ws(("exact", M, K), nb)
        val = torch.empty((M, K), dtype=torch.float32, device=self.device)
        idx = torch.empty((M, K), dtype=torch.int32, device=self.device)
        with torch.cuda.device(self.device):
            check(lib.knn_search_exact(*self._args(), q.data_ptr(), M, K, val.data_ptr(),
                                       idx.data_ptr(), ws.data_ptr(), ws.numel(),
                                       _stream(stream)), "knn_search_exact")
        return val, idx

    def partial_reduce(self, q, L, stream=None, bins="mod"):
        """Alg. 1 alone: (V, A), each M x L (internal scores, indices)."""
        q = q.contiguous()
        M = q.shape[0]
        lib = _lib.get()
        nb = lib.knn_partial_reduce_workspace(self.N, self.D, DTYPE[self.dtype],
                                              METRIC[self.metric], M, L, BINS[bins])
        if nb == 0:
            raise ValueError("invalid partial-reduce arguments")
        ws = self._get_ws(("pr", M, L, bins), nb)
        V = torch.empty((M, L), dtype=torch.float32, device=self.device)
        A = torch.empty((M, L), dtype=torch.int32, device=self.device)
        a = self._args()
        with torch.cuda.device(self.device):
            check(lib.knn_partial_reduce(a[0], a[1], a[2], self.N, self.D, a[6], a[7],
                                         q.data_ptr(), M, L, BINS[bins], V.data_ptr(),
                                         A.data_ptr(), ws.data_ptr(), ws.numel(),
                                         _stream(stream)), "knn_partial_reduce")
        return V, A

    def backward(self, q, idx, grad_val, want_dq=True, want_dx=True, deterministic=False,
                 x_f32=None, stream=None, dx=None, zero_dx=True, atomic=False):
        """Gradient of sum(grad_val * value(q_i, x_idx)) w.r.t. q and the rows.

        dx: an N x D float32 CUDA tensor to write into (default: a new one);
        zero_dx=False adds into it instead of writing zeros over it first
        (for a caller whose dx is already zero, or who accumulates).
        A workspace is passed, so a zero-filled dx is written row by row in
        entry order (bit-reproducible), as is every dx with deterministic=True;
        atomic=True (with deterministic=False) passes none, so the library
        zero-fills and adds with FP32 atomics instead."""
        q = q.contiguous()
        idx = idx.contiguous()
        grad_val = grad_val.contiguous().float()
        M, K = idx.shape
        lib = _lib.get()
        xf = x_f32 if x_f32 is not None else self.f32
        dq = torch.empty((M, self.D), dtype=torch.float32, device=self.device) if want_dq else None
        if want_dx and dx is None:
            dx = torch.empty((self.N, self.D), dtype=torch.float32, device=self.device)
            zero_dx = True
        elif not want_dx:
            dx = None
        elif not (dx.is_cuda and dx.dtype == torch.float32 and dx.is_contiguous()
                  and tuple(dx.shape) == (self.N, self.D)):
            raise ValueError("dx must be a contiguous N x D float32 CUDA tensor")
        if atomic and deterministic:
            raise ValueError("atomic=True is the non-deterministic mode")
        nb = lib.knn_backward_workspace(self.N, self.D, M, K, int(deterministic))
        ws = self._get_ws(("bwd", M, K), nb) if (nb and want_dx and not atomic) else None
        with torch.cuda.device(self.device):
            check(lib.knn_backward(self.lp.data_ptr(), _ptr(self.scale), _ptr(xf), self.N, self.D,
                                   DTYPE[self.dtype], METRIC[self.metric], q.data_ptr(), M, K,
                                   idx.data_ptr(), grad_val.data_ptr(), _ptr(dq), _ptr(dx),
                                   int(bool(zero_dx)), int(deterministic), _ptr(ws),
                                   ws.numel() if ws is not None else 0, _stream(stream)),
                  "knn_backward")
        return dq, dx


class OwnedDatabase:
    """A database held by the library (knn_db_create): the prepared buffers
    live in device memory the library allocated, until close()."""

    def __init__(self, x, metric="l2", dtype="bf16", keep_f32=True, stream=None):
        import ctypes
        if not (x.is_cuda and x.dtype == torch.float32 and x.dim() == 2):
            raise ValueError("x must be a 2-D float32 CUDA tensor")
        x = x.contiguous()
        self.N, self.D = x.shape
        self.metric, self.dtype, self.device = metric, dtype, x.device
        h = ctypes.c_void_p()
        with torch.cuda.device(x.device):
            check(_lib.get().knn_db_create(x.data_ptr(), self.N, self.D, METRIC[metric],
                                           DTYPE[dtype], int(bool(keep_f32)), _stream(stream),
                                           ctypes.byref(h)), "knn_db_create")
        self.handle = h
        self._ws = None

    def search(self, q, K, L=None, recall_target=0.95, rerank=2, stream=None, bins="mod"):
        q = q.contiguous()
        M = q.shape[0]
        L = int(L) if L else plan_bins(self.N, K, recall_target)
        lib = _lib.get()
        nb = lib.knn_db_search_workspace(self.handle, M, K, L, BINS[bins], recall_target, rerank)
        if nb == 0:
            raise ValueError("invalid search arguments")
        if self._ws is None or self._ws.numel() < nb:
            self._ws = _workspace(nb, self.device)
        val = torch.empty((M, K), dtype=torch.float32, device=self.device)
        idx = torch.empty((M, K), dtype=torch.int32, device=self.device)
        with torch.cuda.device(self.device):
            check(lib.knn_db_search(self.handle, q.data_ptr(), M, K, L, BINS[bins], recall_target,
                                    rerank, val.data_ptr(), idx.data_ptr(), self._ws.data_ptr(),
                                    self._ws.numel(), _stream(stream)), "knn_db_search")
        return val, idx

    def close(self):
        if self.handle is not None and self.handle.value:
            with torch.cuda.device(self.device):
                check(_lib.get().knn_db_destroy(self.handle), "knn_db_destroy")
        self.handle = None


def approx_max_k(scores, K, L=None, recall_target=0.95, bins="mod", is_min=False,
                 aggregate_to_topk=True, planning_size=0, stream=None):
    """The approx_max_k / approx_min_k operator (knn_approx_max_k) on an M x N
    FP32 or BF16 CUDA score matrix. Returns (values, indices): M x K best
    first with aggregate_to_topk, else M x L bin winners in bin order."""
    if scores.dim() != 2 or not scores.is_cuda or scores.dtype not in (torch.float32,
                                                                        torch.bfloat16):
        raise ValueError("scores must be a 2-D float32 or bfloat16 CUDA tensor")
    S = scores.contiguous()
    M, N = S.shape
    dt = DTYPE["f32"] if S.dtype == torch.float32 else DTYPE["bf16"]
    lib = _lib.get()
    Lr = int(L) if L else 0
    nb = lib.knn_approx_max_k_workspace(M, N, int(K), Lr, int(planning_size), recall_target,
                                        int(bool(aggregate_to_topk)))
    if nb == 0:
        raise ValueError("invalid approx_max_k arguments (M=%d N=%d K=%d L=%d)" % (M, N, K, Lr))
    if not Lr:
        Lr = min(plan_bins(planning_size or N, K, recall_target), N)
    width = int(K) if aggregate_to_topk else Lr
    val = torch.empty((M, width), dtype=torch.float32, device=S.device)
    idx = torch.empty((M, width), dtype=torch.int32, device=S.device)
    ws = _workspace(nb, S.device)
    with torch.cuda.device(S.device):
        check(lib.knn_approx_max_k(S.data_ptr(), dt, M, N, int(K), Lr, int(planning_size),
                                   recall_target, BINS[bins], int(bool(is_min)),
                                   int(bool(aggregate_to_topk)), val.data_ptr(), idx.data_ptr(),
                                   ws.data_ptr(), ws.numel(), _stream(stream)),
              "knn_approx_max_k")
    return val, idx


def sync_status():
    check(_lib.get().knn_sync_status(), "knn_sync_status")
