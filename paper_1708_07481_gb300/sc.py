"""ctypes binding of libsc_gb300.so (include/sc.h), one Python function per C entry point.

Argument marshalling only: arrays are checked for dtype/contiguity and passed as pointers;
every step of the computation runs in the library's CUDA kernels.  Device arrays may be
passed as torch CUDA tensors (``on_device`` is inferred).  Loading fails loudly when the
library has not been built (run ``python -m paper_1708_07481_gb300.build``); there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsc_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "sc.h")

SC_OK, SC_EINVAL, SC_ENOMEM, SC_EBREAKDOWN, SC_ENOTCONV, SC_ETIMEOUT, SC_ECUDA, SC_EAGAIN = (
    0, -1, -2, -3, -4, -5, -6, -7)
SC_PREC_MIXED, SC_PREC_FP32, SC_PREC_FP64, SC_PREC_MIXED_DD = 0, 1, 2, 3
SC_SYM_LOGICAL, SC_SYM_ALGEBRAIC = 0, 1
SC_MAX_K = 512
_NAMES = {0: "SC_OK", -1: "SC_EINVAL", -2: "SC_ENOMEM", -3: "SC_EBREAKDOWN", -4: "SC_ENOTCONV",
          -5: "SC_ETIMEOUT", -6: "SC_ECUDA", -7: "SC_EAGAIN"}


class ScError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class LobpcgOpts(C.Structure):
    _fields_ = [("iters", C.c_int), ("tol_abs", C.c_double), ("tol_lock", C.c_double),
                ("prec", C.c_int), ("seed", C.c_uint64), ("cold", C.c_int), ("precond", C.c_int)]


SC_PRECOND_NONE, SC_PRECOND_JACOBI = 0, 1


class Request(C.Structure):
    _fields_ = [("kind", C.c_int), ("graph_id", C.c_int), ("n", C.c_int32), ("m", C.c_int64),
                ("src", C.c_void_p), ("dst", C.c_void_p), ("K", C.c_int), ("k", C.c_int),
                ("iters", C.c_int), ("kmeans_iters", C.c_int), ("prec", C.c_int),
                ("tol_abs", C.c_double), ("seed", C.c_uint64)]


SC_REQ_COLD, SC_REQ_DELTA = 0, 1


class EigInfo(C.Structure):
    _fields_ = [("K", C.c_int), ("iters_done", C.c_int), ("fallbacks", C.c_int),
                ("converged", C.c_int), ("lambda_", C.c_double * SC_MAX_K),
                ("resid", C.c_double * SC_MAX_K), ("ms", C.c_float), ("kernels", C.c_uint64),
                ("dropped", C.c_int)]

    def as_dict(self):
        K = self.K
        return dict(K=K, iters_done=self.iters_done, fallbacks=self.fallbacks,
                    converged=self.converged, lam=np.array(self.lambda_[:K]),
                    resid=np.array(self.resid[:K]), ms=float(self.ms), kernels=int(self.kernels),
                    dropped=int(self.dropped))


_lib = None


def lib():
    """Load the library once; raise if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with python -m paper_1708_07481_gb300.build")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    sig = {
        "sc_ctx_create": ([C.POINTER(vp), C.c_int, vp, C.c_size_t], C.c_int),
        "sc_ctx_destroy": ([vp], None),
        "sc_last_error": ([vp], C.c_char_p),
        "sc_ctx_bytes_in_use": ([vp], C.c_size_t),
        "sc_ctx_bytes_peak": ([vp], C.c_size_t),
        "sc_ctx_kernel_launches": ([vp], u64),
        "sc_ctx_graph_replays": ([vp], u64),
        "sc_ctx_batch_lockstep_passes": ([vp], u64),
        "sc_debug_inject": ([vp, C.c_int, C.c_longlong], C.c_int),
        "sc_profile_begin": ([vp, C.c_char_p], C.c_int),
        "sc_profile_end": ([vp, C.c_char_p, C.c_size_t], C.c_int),
        "sc_build_laplacian": ([vp, i32, i64, vp, vp, vp, C.c_int, C.c_int, C.POINTER(vp)], C.c_int),
        "sc_graph_info": ([vp, C.POINTER(i32), C.POINTER(i64), C.POINTER(dbl)], C.c_int),
        "sc_graph_copy_csr": ([vp, vp, vp, vp, vp], C.c_int),
        "sc_graph_destroy": ([vp], None),
        "sc_lap_apply": ([vp, vp, C.c_int, C.c_int, vp, vp, C.c_int], C.c_int),
        "sc_lobpcg": ([vp, vp, C.c_int, C.POINTER(LobpcgOpts), vp, i32, vp, C.POINTER(EigInfo)], C.c_int),
        "sc_lobpcg64": ([vp, vp, C.c_int, C.POINTER(LobpcgOpts), vp, i32, vp, C.POINTER(EigInfo)], C.c_int),
        "sc_embed_rows": ([vp, vp, i32, C.c_int, vp, C.c_int], C.c_int),
        "sc_kmeans": ([vp, vp, i32, C.c_int, C.c_int, C.c_int, u64, vp, C.c_int, vp, vp, vp,
                       C.POINTER(dbl), C.POINTER(C.c_int)], C.c_int),
        "sc_cpqr_assign": ([vp, vp, i32, C.c_int, C.c_int, vp, vp], C.c_int),
        "sc_eigengap": ([vp, C.c_int, dbl, dbl, C.POINTER(C.c_int)], C.c_int),
        "sc_partition": ([vp, vp, C.c_int, C.c_int, C.POINTER(LobpcgOpts), C.c_int, vp,
                          C.POINTER(EigInfo)], C.c_int),
        "sc_stream_update": ([vp, vp, i32, i64, vp, vp, vp, C.c_int], C.c_int),
        "sc_gram": ([vp, C.c_int, i64, C.c_int, C.c_int, vp, i64, vp, i64, vp, C.c_int], C.c_int),
        "sc_rr_solve": ([vp, C.c_int, C.c_int, C.c_int, vp, vp, vp], C.c_int),
        "sc_tall_update": ([vp, C.c_int, i64, C.c_int, C.c_int, vp, i64, vp, vp, i64, dbl, vp, i64,
                            C.c_int], C.c_int),
        "sc_lobpcg_batch": ([vp, C.c_int, vp, vp, vp, vp], C.c_int),
        "sc_lobpcg_blocks": ([vp, vp, C.c_int, C.c_int, C.POINTER(LobpcgOpts), vp, vp,
                              C.POINTER(EigInfo)], C.c_int),
        "sc_partition_batch": ([vp, C.c_int, vp, vp, vp, vp, C.c_int, vp, vp], C.c_int),
        "sc_server_create": ([vp, C.c_int, C.c_int, C.POINTER(vp)], C.c_int),
        "sc_server_submit": ([vp, C.POINTER(Request), C.POINTER(u64)], C.c_int),
        "sc_server_poll": ([vp, u64, vp, i32, C.POINTER(EigInfo), C.POINTER(dbl)], C.c_int),
        "sc_server_wait": ([vp, u64, C.c_int, vp, i32, C.POINTER(EigInfo), C.POINTER(dbl)], C.c_int),
        "sc_server_stats": ([vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(u64)], C.c_int),
        "sc_server_destroy": ([vp], None),
        "sc_gram_static": ([i64, C.c_int, C.c_int, vp, i64, vp, i64, vp, vp], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def declared_symbols(header: str = HEADER) -> list[str]:
    """Entry points declared in include/sc.h."""
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sc_[a-z0-9_]+)\s*\(", txt)))


# ---------------------------------------------------------------------------------------


def _ptr(a):
    """(pointer, on_device) of a numpy array or a torch tensor."""
    if a is None:
        return None, 0
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr()), int(bool(a.is_cuda))
    return a.ctypes.data_as(C.c_void_p), 0


def _np(a, dtype):
    if hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=dtype)


class Ctx:
    def __init__(self, device=0, stream=None, budget=0):
        import weakref

        self.h = C.c_void_p()
        self.children = weakref.WeakSet()  # graphs and servers that must go first
        s = C.c_void_p(stream) if stream else None
        rc = lib().sc_ctx_create(C.byref(self.h), device, s, budget)
        if rc != SC_OK:
            raise ScError(rc, "sc_ctx_create failed")

    def check(self, rc):
        if rc != SC_OK:
            raise ScError(rc, lib().sc_last_error(self.h).decode())
        return rc

    def close(self):
        if self.h:
            for ch in list(self.children):
                ch.close()
            lib().sc_ctx_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def bytes_in_use(self):
        return lib().sc_ctx_bytes_in_use(self.h)

    def bytes_peak(self):
        """High-water mark since the previous call (then reset to the current use)."""
        return lib().sc_ctx_bytes_peak(self.h)

    @property
    def launches(self):
        return lib().sc_ctx_kernel_launches(self.h)

    @property
    def graph_replays(self):
        return lib().sc_ctx_graph_replays(self.h)

    @property
    def lockstep_passes(self):
        return lib().sc_ctx_batch_lockstep_passes(self.h)


class Graph:
    def __init__(self, ctx, h):
        self.ctx, self.h = ctx, h
        ctx.children.add(self)

    def close(self):
        if self.h and self.ctx.h:
            lib().sc_graph_destroy(self.h)
        self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sc_ctx_create(device=0, stream=None, budget=0) -> Ctx:
    return Ctx(device, stream, budget)


SC_INJECT_NONE, SC_INJECT_WAIT_TIMEOUT, SC_INJECT_P_BREAKDOWN = 0, 1, 2


def sc_debug_inject(ctx: Ctx, kind, arg=0):
    """Arm (or with SC_INJECT_NONE disarm) an injected failure on the context (tests only)."""
    ctx.check(lib().sc_debug_inject(ctx.h, int(kind), int(arg)))


def sc_profile_begin(ctx: Ctx, kernels: str = "*"):
    ctx.check(lib().sc_profile_begin(ctx.h, kernels.encode()))


def sc_profile_end(ctx: Ctx) -> dict:
    """-> {kernel: (launches, total device ms)} since sc_profile_begin."""
    buf = C.create_string_buffer(1 << 16)
    ctx.check(lib().sc_profile_end(ctx.h, buf, len(buf)))
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


def sc_build_laplacian(ctx: Ctx, n, src, dst, w=None, sym=SC_SYM_LOGICAL) -> Graph:
    src, dst = _np(src, np.int32), _np(dst, np.int32)
    w = None if w is None else _np(w, np.float32)
    ps, dev = _ptr(src)
    pd, _ = _ptr(dst)
    pw, _ = _ptr(w)
    m = int(src.shape[0])
    h = C.c_void_p()
    ctx.check(lib().sc_build_laplacian(ctx.h, n, m, ps, pd, pw, sym, dev, C.byref(h)))
    return Graph(ctx, h)


def sc_graph_info(g: Graph):
    n, nnz, dm = C.c_int32(), C.c_int64(), C.c_double()
    g.ctx.check(lib().sc_graph_info(g.h, C.byref(n), C.byref(nnz), C.byref(dm)))
    return n.value, nnz.value, dm.value


def sc_graph_copy_csr(g: Graph):
    n, nnz, _ = sc_graph_info(g)
    rp = np.empty(n + 1, np.int32)
    ci = np.empty(max(nnz, 1), np.int32)
    val = np.empty(max(nnz, 1), np.float32)
    deg = np.empty(n, np.float64)
    g.ctx.check(lib().sc_graph_copy_csr(g.h, _ptr(rp)[0], _ptr(ci)[0], _ptr(val)[0], _ptr(deg)[0]))
    return rp, ci[:nnz], val[:nnz], deg


def sc_lap_apply(ctx: Ctx, g: Graph, V, prec=SC_PREC_FP32):
    dt = np.float64 if prec == SC_PREC_FP64 else np.float32
    V = _np(V, dt)
    if hasattr(V, "data_ptr"):
        import torch
        Y = torch.empty_like(V)
    else:
        Y = np.empty_like(V)
    pv, dev = _ptr(V)
    ctx.check(lib().sc_lap_apply(ctx.h, g.h, int(V.shape[1]), prec, pv, _ptr(Y)[0], dev))
    return Y


def sc_lobpcg(ctx: Ctx, g: Graph, K, iters=20, tol_abs=0.0, tol_lock=0.0, prec=SC_PREC_MIXED,
              seed=0, cold=0, X0=None, x0_rows=0, want_X=True, precond=SC_PRECOND_NONE):
    o = LobpcgOpts(iters, tol_abs, tol_lock, prec, seed, cold, precond)
    info = EigInfo()
    n = sc_graph_info(g)[0]
    X = np.empty((n, K), np.float32) if want_X else None
    x0 = None if X0 is None else np.ascontiguousarray(X0, dtype=np.float32)
    rc = lib().sc_lobpcg(ctx.h, g.h, K, C.byref(o), _ptr(x0)[0], int(x0_rows), _ptr(X)[0],
                         C.byref(info))
    d = info.as_dict()
    if rc != SC_OK:
        err = ScError(rc, lib().sc_last_error(ctx.h).decode())
        err.info = d
        raise err
    return d["lam"], d["resid"], X, d


def sc_lobpcg64(ctx: Ctx, g: Graph, K, iters=20, tol_abs=0.0, tol_lock=0.0,
                prec=SC_PREC_FP64, seed=0, cold=0, X0=None, x0_rows=0, want_X=True,
                precond=SC_PRECOND_NONE):
    """sc_lobpcg with an FP64 start block and an FP64 result block (host arrays)."""
    o = LobpcgOpts(iters, tol_abs, tol_lock, prec, seed, cold, precond)
    info = EigInfo()
    n = sc_graph_info(g)[0]
    X = np.empty((n, K), np.float64) if want_X else None
    x0 = None if X0 is None else np.ascontiguousarray(X0, dtype=np.float64)
    rc = lib().sc_lobpcg64(ctx.h, g.h, K, C.byref(o), _ptr(x0)[0], int(x0_rows), _ptr(X)[0],
                           C.byref(info))
    d = info.as_dict()
    if rc != SC_OK:
        err = ScError(rc, lib().sc_last_error(ctx.h).decode())
        err.info = d
        raise err
    return d["lam"], d["resid"], X, d


def sc_embed_rows(ctx: Ctx, X):
    X = _np(X, np.float32)
    if hasattr(X, "data_ptr"):
        import torch
        E = torch.empty_like(X)
    else:
        E = np.empty_like(X)
    px, dev = _ptr(X)
    ctx.check(lib().sc_embed_rows(ctx.h, px, int(X.shape[0]), int(X.shape[1]), _ptr(E)[0], dev))
    return E


def sc_kmeans(ctx: Ctx, E, k, iters=50, seed=0, init_idx=None):
    E = _np(E, np.float32)
    n, d = int(E.shape[0]), int(E.shape[1])
    labels = np.empty(n, np.int32)
    cent = np.empty((k, d), np.float32)
    seeds = np.empty(k, np.int32)
    inertia = C.c_double()
    ran = C.c_int()
    init = None if init_idx is None else np.ascontiguousarray(init_idx, dtype=np.int32)
    pe, dev = _ptr(E)
    ctx.check(lib().sc_kmeans(ctx.h, pe, n, d, k, iters, seed, _ptr(init)[0], dev, _ptr(labels)[0],
                              _ptr(cent)[0], _ptr(seeds)[0], C.byref(inertia), C.byref(ran)))
    return labels, cent, seeds, inertia.value, ran.value


def sc_cpqr_assign(ctx: Ctx, Y):
    """Labels and pivot rows of the eigenvector block Y (n x K) by QR with column pivoting."""
    Y = _np(Y, np.float32)
    n, K = int(Y.shape[0]), int(Y.shape[1])
    labels = np.empty(n, np.int32)
    piv = np.empty(K, np.int32)
    py, dev = _ptr(Y)
    ctx.check(lib().sc_cpqr_assign(ctx.h, py, n, K, dev, _ptr(labels)[0], _ptr(piv)[0]))
    return labels, piv


def sc_eigengap(lam, ratio=4.0, floor=0.0):
    """Cluster count from the first significantly large increment of the eigenvalues lam
    (host arithmetic in the library); 0 when there is no such increment."""
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    k = C.c_int(0)
    rc = lib().sc_eigengap(_ptr(lam)[0], int(lam.size), float(ratio), float(floor), C.byref(k))
    if rc != SC_OK:
        raise ScError(rc, "sc_eigengap: invalid argument")
    return k.value


def sc_partition(ctx: Ctx, g: Graph, K, k, iters=20, kmeans_iters=50, prec=SC_PREC_MIXED,
                 seed=0, tol_abs=0.0, tol_lock=0.0, cold=1, precond=SC_PRECOND_NONE):
    o = LobpcgOpts(iters, tol_abs, tol_lock, prec, seed, cold, precond)
    info = EigInfo()
    n = sc_graph_info(g)[0]
    labels = np.empty(n, np.int32)
    ctx.check(lib().sc_partition(ctx.h, g.h, K, k, C.byref(o), kmeans_iters, _ptr(labels)[0],
                                 C.byref(info)))
    return labels, info.as_dict()


def sc_stream_update(ctx: Ctx, g: Graph, n_new, src, dst, w=None):
    src, dst = _np(src, np.int32), _np(dst, np.int32)
    w = None if w is None else _np(w, np.float32)
    ps, dev = _ptr(src)
    ctx.check(lib().sc_stream_update(ctx.h, g.h, n_new, int(src.shape[0]), ps, _ptr(dst)[0],
                                     _ptr(w)[0], dev))


def sc_gram(ctx: Ctx, A, B, prec=SC_PREC_FP32):
    dt = np.float64 if prec == SC_PREC_FP64 else np.float32
    A, B = _np(A, dt), _np(B, dt)
    n, a = int(A.shape[0]), int(A.shape[1])
    b = int(B.shape[1])
    Cm = np.empty((a, b), np.float64)
    pa, dev = _ptr(A)
    ctx.check(lib().sc_gram(ctx.h, prec, n, a, b, pa, a, _ptr(B)[0], b, _ptr(Cm)[0], dev))
    return Cm


def sc_tall_update(ctx: Ctx, A, W, Cin=None, beta=1.0, prec=SC_PREC_MIXED):
    """out = beta Cin + A W (host numpy arrays; float64 with SC_PREC_FP64, else float32)."""
    dt = np.float64 if prec == SC_PREC_FP64 else np.float32
    A, W = _np(A, dt), _np(W, dt)
    n, a = int(A.shape[0]), int(A.shape[1])
    b = int(W.shape[1])
    Cin = None if Cin is None else _np(Cin, dt)
    out = np.empty((n, b), dt)
    ctx.check(lib().sc_tall_update(ctx.h, prec, n, a, b, _ptr(A)[0], a, _ptr(W)[0], _ptr(Cin)[0],
                                   b, float(beta), _ptr(out)[0], b, 0))
    return out


def sc_rr_solve(ctx: Ctx, G, K, prec=SC_PREC_FP32):
    G = np.ascontiguousarray(G, dtype=np.float64)
    m = G.shape[0]
    th = np.empty(K, np.float64)
    Y = np.empty((m, K), np.float64)
    ctx.check(lib().sc_rr_solve(ctx.h, prec, m, K, _ptr(G)[0], _ptr(th)[0], _ptr(Y)[0]))
    return th, Y


def sc_lobpcg_blocks(ctx: Ctx, g: Graph, K, nb, iters=20, tol_abs=0.0, tol_lock=0.0,
                     prec=SC_PREC_MIXED, seed=0, X0=None, precond=SC_PRECOND_NONE):
    """Hard locking: the K smallest eigenpairs nb at a time; returns (lam, resid, X, info)."""
    o = LobpcgOpts(iters, tol_abs, tol_lock, prec, seed, 1, precond)
    info = EigInfo()
    n = sc_graph_info(g)[0]
    X = np.empty((n, K), np.float32)
    x0 = None if X0 is None else np.ascontiguousarray(X0, dtype=np.float32)
    ctx.check(lib().sc_lobpcg_blocks(ctx.h, g.h, K, nb, C.byref(o), _ptr(x0)[0], _ptr(X)[0],
                                     C.byref(info)))
    d = info.as_dict()
    return d["lam"], d["resid"], X, d


def sc_lobpcg_batch(ctx: Ctx, graphs, K, iters=20, tol_abs=0.0, prec=SC_PREC_MIXED, seeds=None,
                    cold=1):
    """Batched LOBPCG over several graphs; returns a list of info dicts."""
    cnt = len(graphs)
    Ks = (C.c_int * cnt)(*([K] * cnt if isinstance(K, int) else K))
    hs = (C.c_void_p * cnt)(*[g.h.value for g in graphs])
    seeds = seeds or [0] * cnt
    opts = (LobpcgOpts * cnt)(*[LobpcgOpts(iters, tol_abs, 0.0, prec, s, cold, 0) for s in seeds])
    infos = (EigInfo * cnt)()
    ctx.check(lib().sc_lobpcg_batch(ctx.h, cnt, hs, Ks, opts, infos))
    return [infos[q].as_dict() for q in range(cnt)]


def sc_partition_batch(ctx: Ctx, graphs, K, k, iters=20, kmeans_iters=50, prec=SC_PREC_MIXED,
                       seeds=None):
    cnt = len(graphs)
    Kl = [K] * cnt if isinstance(K, int) else list(K)
    kl = [k] * cnt if isinstance(k, int) else list(k)
    seeds = seeds or [0] * cnt
    outs = [np.empty(sc_graph_info(g)[0], np.int32) for g in graphs]
    lp = (C.c_void_p * cnt)(*[o.ctypes.data for o in outs])
    hs = (C.c_void_p * cnt)(*[g.h.value for g in graphs])
    opts = (LobpcgOpts * cnt)(*[LobpcgOpts(iters, 0.0, 0.0, prec, s, 1, 0) for s in seeds])
    infos = (EigInfo * cnt)()
    ctx.check(lib().sc_partition_batch(ctx.h, cnt, hs, (C.c_int * cnt)(*Kl), (C.c_int * cnt)(*kl),
                                       opts, kmeans_iters, lp, infos))
    return outs, [infos[q].as_dict() for q in range(cnt)]


class Server:
    """Continuous-batching partition server (thread-safe)."""

    def __init__(self, ctx: Ctx, max_slots=8, queue_cap=64):
        self.ctx = ctx
        self.h = C.c_void_p()
        ctx.check(lib().sc_server_create(ctx.h, max_slots, queue_cap, C.byref(self.h)))
        ctx.children.add(self)

    def submit(self, kind, graph_id, n, src, dst, K, k, iters=20, kmeans_iters=50,
               prec=SC_PREC_MIXED, tol_abs=0.0, seed=0):
        src = np.ascontiguousarray(src, np.int32)
        dst = np.ascontiguousarray(dst, np.int32)
        r = Request(kind, graph_id, n, src.shape[0], src.ctypes.data, dst.ctypes.data, K, k, iters,
                    kmeans_iters, prec, tol_abs, seed)
        t = C.c_uint64()
        rc = lib().sc_server_submit(self.h, C.byref(r), C.byref(t))
        if rc != SC_OK:
            raise ScError(rc, "sc_server_submit")
        return t.value

    def wait(self, ticket, n_cap, timeout_ms=600000):
        labels = np.empty(max(n_cap, 1), np.int32)
        info = EigInfo()
        lat = C.c_double()
        rc = lib().sc_server_wait(self.h, ticket, timeout_ms, labels.ctypes.data, n_cap,
                                  C.byref(info), C.byref(lat))
        return rc, labels[:n_cap], info.as_dict(), lat.value

    def stats(self):
        a, q, d = C.c_int(), C.c_int(), C.c_uint64()
        lib().sc_server_stats(self.h, C.byref(a), C.byref(q), C.byref(d))
        return a.value, q.value, d.value

    def close(self):
        if self.h and self.ctx.h:
            lib().sc_server_destroy(self.h)
        self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sc_server_create(ctx: Ctx, max_slots=8, queue_cap=64) -> Server:
    return Server(ctx, max_slots, queue_cap)


def sc_gram_static(A, B, C_out, stream=None):
    """C_out = A' B without any device allocation (see include/sc.h): A (n x a), B (n x b) are
    float32 CUDA tensors, C_out an (a x b) float64 CUDA tensor; issued on `stream` (a
    cudaStream_t handle; None = torch's current stream) without waiting for it."""
    import torch

    if A.dtype != torch.float32 or B.dtype != torch.float32 or C_out.dtype != torch.float64:
        raise TypeError("sc_gram_static: A, B float32 and C_out float64 expected")
    if not (A.is_cuda and B.is_cuda and C_out.is_cuda):
        raise ValueError("sc_gram_static: device tensors expected")
    if A.dim() != 2 or B.dim() != 2 or A.shape[0] != B.shape[0]:
        raise ValueError("sc_gram_static: A (n x a) and B (n x b) expected")
    n, a = int(A.shape[0]), int(A.shape[1])
    b = int(B.shape[1])
    if (A.stride(1) != 1 and a > 1) or (B.stride(1) != 1 and b > 1) or \
            tuple(C_out.shape) != (a, b) or not C_out.is_contiguous():
        raise ValueError("sc_gram_static: row-major A, B and a contiguous (a x b) C_out expected")
    if stream is None:
        stream = torch.cuda.current_stream(A.device).cuda_stream
    rc = lib().sc_gram_static(n, a, b, C.c_void_p(A.data_ptr()), int(A.stride(0)),
                              C.c_void_p(B.data_ptr()), int(B.stride(0)),
                              C.c_void_p(C_out.data_ptr()), C.c_void_p(stream) if stream else None)
    if rc != SC_OK:
        raise ScError(rc, "sc_gram_static")
