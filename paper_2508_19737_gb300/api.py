"""ctypes binding over the C-ABI of libigp.so (include/igp.h), same names.

Argument marshalling only: every step of the FFP runs in the library's CUDA
kernels. Buffers may be numpy arrays (host) or torch tensors (host or CUDA);
the library itself tells host from device pointers. Raises IgpError on a
non-zero status and RuntimeError if the library has not been built.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libigp.so")

IGP_OK = 0
IGP_E_INVAL = 1
IGP_E_NOMEM = 2
IGP_E_CUDA = 3
IGP_E_TIMEOUT = 4
IGP_E_BUSY = 5
IGP_E_NOTREADY = 6
IGP_E_CANCELLED = 7
IGP_E_UNSUPPORTED = 8

IGP_STORE_F32 = 0
IGP_STORE_BF16 = 1

IGP_GATHER_AUTO = 0
IGP_GATHER_LSU = 1
IGP_GATHER_BULK = 2
IGP_GATHER_TMA4 = 3
GATHER = {"auto": IGP_GATHER_AUTO, "lsu": IGP_GATHER_LSU, "bulk": IGP_GATHER_BULK, "tma4": IGP_GATHER_TMA4}

IGP_PHASE_DINV = 0
IGP_PHASE_THETA = 1
IGP_PHASE_LAYER = 2
IGP_PHASE_OUTPUT = 3
IGP_PHASE_BUILD = 4
IGP_NUM_PHASES = 5
PHASE_NAMES = ["dinv", "theta", "layer", "output", "build"]

STORAGE = {"f32": IGP_STORE_F32, "bf16": IGP_STORE_BF16}


class IgpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"igp status {status}: {msg}")
        self.status = status


class EmbedOpts(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_double),
        ("theta", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("x_scale", ctypes.c_double),
        ("znorm_ddof", ctypes.c_int32),
        ("storage", ctypes.c_int32),
        ("out_row_l2", ctypes.c_int32),
        ("chunk_cols", ctypes.c_int32),
        ("gather", ctypes.c_int32),
        ("reserved_test", ctypes.c_int32),
        ("out_row_begin", ctypes.c_int32),
        ("host_async", ctypes.c_int32),
        ("x_in", ctypes.c_void_p),
        ("profile", ctypes.c_void_p),
    ]


class ServerOpts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_queue", ctypes.c_int32), ("reserve_bytes", ctypes.c_int64),
                ("device", ctypes.c_int32), ("batch_rows", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("keep", ctypes.c_int32), ("graph_id", ctypes.c_int64),
                ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("M", ctypes.c_int64), ("N", ctypes.c_int32),
                ("L", ctypes.c_int32), ("tau", ctypes.c_double), ("d", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("seed", ctypes.c_uint64), ("opts", EmbedOpts),
                ("out", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "failed", "cancelled", "queued", "running",
                                              "resident_graphs", "admitted_bytes", "budget_bytes")] + \
               [("latency_p50_s", ctypes.c_double), ("latency_p99_s", ctypes.c_double),
                ("resident_bytes", ctypes.c_int64), ("batches", ctypes.c_int64), ("batched", ctypes.c_int64)]


IGP_REQ_EMBED = 0
IGP_REQ_APPEND = 1
REQ_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "cancelled"}

_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "igp_version": (ctypes.c_char_p, []),
    "igp_last_error": (ctypes.c_char_p, []),
    "igp_launch_count": (ctypes.c_int64, []),
    "igp_alloc_count": (ctypes.c_int64, []),
    "igp_embed_opts_init": (None, [ctypes.POINTER(EmbedOpts)]),
    "igp_graph_build": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "igp_graph_build_profiled": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "igp_graph_append": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_int32, ctypes.c_void_p]),
    "igp_graph_info": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]),
    "igp_graph_export": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "igp_graph_import": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                          ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "igp_degree_factors": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "igp_graph_free": (None, [ctypes.c_void_p]),
    "igp_graph_sync": (ctypes.c_int32, [ctypes.c_void_p]),
    "igp_generate_x": (ctypes.c_int32, [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "igp_embed": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER(EmbedOpts), ctypes.c_void_p]),
    "igp_embed_noalloc": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_double,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p,
                                           ctypes.POINTER(EmbedOpts), ctypes.c_void_p]),
    "igp_clusterer_create": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_void_p)]),
    "igp_clusterer_fit": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "igp_clusterer_predict": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.c_void_p]),
    "igp_clusterer_info": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p]),
    "igp_clusterer_free": (None, [ctypes.c_void_p]),
    "igp_batch_create": (ctypes.c_int32, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "igp_batch_info": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                                        ctypes.c_void_p]),
    "igp_batch_sync": (ctypes.c_int32, [ctypes.c_void_p]),
    "igp_batch_embed": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(EmbedOpts),
                                         ctypes.c_void_p]),
    "igp_batch_free": (None, [ctypes.c_void_p]),
    "igp_server_opts_init": (None, [ctypes.POINTER(ServerOpts)]),
    "igp_server_create": (ctypes.c_int32, [ctypes.POINTER(ServerOpts), ctypes.POINTER(ctypes.c_void_p)]),
    "igp_server_destroy": (None, [ctypes.c_void_p]),
    "igp_submit": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "igp_poll": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_double)]),
    "igp_wait": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_double)]),
    "igp_cancel": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64]),
    "igp_server_forget": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64]),
    "igp_server_release": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int64]),
    "igp_server_get_stats": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ServerStats)]),
    "igp_profile_create": (ctypes.c_int32, [ctypes.POINTER(ctypes.c_void_p)]),
    "igp_profile_free": (None, [ctypes.c_void_p]),
    "igp_profile_read": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int64)]),
}


def lib():
    """Load libigp.so (once). Raises if it has not been built: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2508_19737_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(status):
    if status != IGP_OK:
        raise IgpError(status, lib().igp_last_error().decode())


def _ptr(x):
    """Raw address of a numpy array or torch tensor (contiguous), or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def version():
    return lib().igp_version().decode()


def launch_count():
    return int(lib().igp_launch_count())


def alloc_count():
    """igp_alloc_count: memory allocations the library has made in this process."""
    return int(lib().igp_alloc_count())


def embed_opts(alpha=1.0, theta=0.1, eps=1e-3, x_scale=0.0, znorm_ddof=1, storage="f32", out_row_l2=False,
               x_in=None, profile=None, chunk_cols=0, gather="auto", reserved_test=0, out_row_begin=0,
               host_async=False):
    o = EmbedOpts()
    lib().igp_embed_opts_init(ctypes.byref(o))
    o.alpha, o.theta, o.eps, o.x_scale = alpha, theta, eps, x_scale
    o.znorm_ddof = znorm_ddof
    o.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    o.out_row_l2 = 1 if out_row_l2 else 0
    o.chunk_cols = int(chunk_cols)
    o.gather = GATHER[gather] if isinstance(gather, str) else int(gather)
    o.reserved_test = int(reserved_test)
    o.out_row_begin = int(out_row_begin)
    o.host_async = 1 if host_async else 0
    o.x_in = _ptr(x_in)
    o.profile = profile.handle if profile is not None else None
    return o


class Profile:
    """Per-phase device time recorded with CUDA events (igp_profile_*)."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(lib().igp_profile_create(ctypes.byref(h)))
        self.handle = h.value

    def read(self):
        ms = (ctypes.c_double * IGP_NUM_PHASES)()
        n = (ctypes.c_int64 * IGP_NUM_PHASES)()
        _check(lib().igp_profile_read(self.handle, ms, n))
        return {PHASE_NAMES[i]: (ms[i], n[i]) for i in range(IGP_NUM_PHASES)}

    def close(self):
        if self.handle:
            lib().igp_profile_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """Owning wrapper of an igp_graph handle."""

    def __init__(self, handle):
        self.handle = handle

    def info(self):
        n = ctypes.c_int32()
        nnz = ctypes.c_int64()
        md = ctypes.c_int32()
        _check(lib().igp_graph_info(self.handle, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(md)))
        return n.value, nnz.value, md.value

    @property
    def N(self):
        return self.info()[0]

    @property
    def nnz(self):
        return self.info()[1]

    def export(self, row_ptr=None, col=None, stream=None):
        """Copy the CSR into the given buffers, or into new numpy arrays if none given."""
        N, nnz, _ = self.info()
        if row_ptr is None and col is None:
            row_ptr = np.empty(N + 1, dtype=np.int32)
            col = np.empty(nnz, dtype=np.int32)
        _check(lib().igp_graph_export(self.handle, _ptr(row_ptr), _ptr(col), _stream(stream)))
        return row_ptr, col

    def append(self, src, dst, N_new, stream=None):
        """igp_graph_append: merge an edge increment (int32 arrays, host or device), growing to N_new."""
        M = int(src.shape[0])
        if int(dst.shape[0]) != M:
            raise ValueError("src and dst differ in length")
        _check(lib().igp_graph_append(self.handle, _ptr(src), _ptr(dst), M, int(N_new), _stream(stream)))

    def sync(self):
        """igp_graph_sync: wait for the handle's work; raises IgpError(IGP_E_TIMEOUT) if a
        device-side wait of the last embed ran out."""
        _check(lib().igp_graph_sync(self.handle))

    def free(self):
        if self.handle:
            lib().igp_graph_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def graph_build(src, dst, N, stream=None, profile=None):
    """igp_graph_build: src/dst int32 (numpy or torch, host or device)."""
    M = int(src.shape[0])
    if int(dst.shape[0]) != M:
        raise ValueError("src and dst differ in length")
    for a in (src, dst):
        if str(a.dtype) not in ("int32", "torch.int32"):
            raise TypeError("edge arrays must be int32")
    h = ctypes.c_void_p()
    if profile is None:
        st = lib().igp_graph_build(_ptr(src), _ptr(dst), M, int(N), _stream(stream), ctypes.byref(h))
    else:
        st = lib().igp_graph_build_profiled(_ptr(src), _ptr(dst), M, int(N), _stream(stream), profile.handle,
                                            ctypes.byref(h))
    _check(st)
    return Graph(h.value)


def graph_import(row_ptr, col, N, validate=True, stream=None):
    """igp_graph_import: a Graph from a CSR (numpy arrays or tensors, host or device)."""
    nnz = int(col.shape[0]) if col is not None else 0
    h = ctypes.c_void_p()
    _check(lib().igp_graph_import(_ptr(row_ptr), _ptr(col) if nnz else None, int(N), nnz, 1 if validate else 0,
                                  _stream(stream), ctypes.byref(h)))
    return Graph(h.value)


def degree_factors(g, tau, eps=1e-3, out=None, stream=None):
    """igp_degree_factors: fp32 D_tau^{-1/2} (numpy array unless `out` is given)."""
    if out is None:
        out = np.empty(g.N, dtype=np.float32)
    _check(lib().igp_degree_factors(g.handle, float(tau), float(eps), _ptr(out), _stream(stream)))
    return out


def generate_x(seed, N, d, x_scale=0.0, out=None, stream=None):
    """igp_generate_x: the Theta igp_embed draws, as fp32 [N, d]."""
    if out is None:
        out = np.empty((N, d), dtype=np.float32)
    _check(lib().igp_generate_x(int(seed) & 0xFFFFFFFFFFFFFFFF, int(N), int(d), float(x_scale), _ptr(out),
                                _stream(stream)))
    return out


def embed(g, tau, L, d, seed, out=None, opts=None, stream=None, **kw):
    """igp_embed: one FFP; returns `out` (a new numpy array if not given) holding rows
    out_row_begin .. N-1 of the embedding (all rows by default)."""
    if opts is None:
        opts = embed_opts(**kw)
    elif kw:
        raise ValueError("give either opts or keyword options")
    if out is None:
        out = np.empty((max(g.N - opts.out_row_begin, 0), d), dtype=np.float32)
    _check(lib().igp_embed(g.handle, float(tau), int(L), int(d), int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(out),
                           ctypes.byref(opts), _stream(stream)))
    return out


def embed_noalloc(row_ptr, col, N, tau, L, d, seed, out, opts=None, stream=None, **kw):
    """igp_embed_noalloc: one FFP on a caller-held device CSR into a device `out`, using only the
    library's fixed scratch array (for callers that must not allocate during the call)."""
    if opts is None:
        opts = embed_opts(**kw)
    elif kw:
        raise ValueError("give either opts or keyword options")
    _check(lib().igp_embed_noalloc(_ptr(row_ptr), _ptr(col), int(N), float(tau), int(L), int(d),
                                   int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(out), ctypes.byref(opts), _stream(stream)))
    return out


class Batch:
    """Owning wrapper of an igp_batch handle (many graphs embedded together)."""

    def __init__(self, graphs, stream=None):
        arr = (ctypes.c_void_p * len(graphs))(*[g.handle for g in graphs])
        h = ctypes.c_void_p()
        _check(lib().igp_batch_create(arr, len(graphs), _stream(stream), ctypes.byref(h)))
        self.handle = h.value

    def info(self):
        G = ctypes.c_int32()
        N = ctypes.c_int32()
        nnz = ctypes.c_int64()
        _check(lib().igp_batch_info(self.handle, ctypes.byref(G), ctypes.byref(N), ctypes.byref(nnz), None))
        offs = np.empty(G.value + 1, dtype=np.int32)
        _check(lib().igp_batch_info(self.handle, None, None, None, offs.ctypes.data))
        return G.value, N.value, nnz.value, offs

    def embed(self, tau, L, d, seeds, out=None, opts=None, stream=None, **kw):
        """igp_batch_embed; seeds: G integers. Returns `out` (N_total x d)."""
        if opts is None:
            opts = embed_opts(**kw)
        elif kw:
            raise ValueError("give either opts or keyword options")
        G, N, _, _ = self.info()
        sd = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
        if sd.size != G:
            raise ValueError("need one seed per graph")
        if out is None:
            out = np.empty((N, d), dtype=np.float32)
        _check(lib().igp_batch_embed(self.handle, float(tau), int(L), int(d), sd.ctypes.data, _ptr(out),
                                     ctypes.byref(opts), _stream(stream)))
        return out

    def sync(self):
        """igp_batch_sync: wait for the last embedding; raises IgpError(IGP_E_TIMEOUT) if a bounded
        device-side wait of its persistent launch ran out."""
        _check(lib().igp_batch_sync(self.handle))

    def free(self):
        if self.handle:
            lib().igp_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Clusterer:
    """Owning wrapper of an igp_clusterer (K-agnostic clustering on the device, BIRCH's leaf level).
    partial_fit / predict follow the interface stream.StreamingPartitioner expects."""

    def __init__(self, d, threshold, batch=1024, max_entries=1 << 20):
        h = ctypes.c_void_p()
        _check(lib().igp_clusterer_create(int(d), float(threshold), int(batch), int(max_entries), ctypes.byref(h)))
        self.handle = h.value
        self.d = int(d)

    def _points(self, E):
        if isinstance(E, np.ndarray):
            E = np.ascontiguousarray(E, dtype=np.float32)
        if E.shape[1] != self.d:
            raise ValueError(f"points must have {self.d} columns")
        return E

    def fit(self, E, labels=None, stream=None):
        """igp_clusterer_fit (a partial fit). Returns the labels (int32 numpy array unless a
        device `labels` buffer is given)."""
        E = self._points(E)
        if labels is None:
            labels = np.empty(E.shape[0], dtype=np.int32)
        _check(lib().igp_clusterer_fit(self.handle, _ptr(E), int(E.shape[0]), _ptr(labels), _stream(stream)))
        return labels

    partial_fit = fit

    def predict(self, E, labels=None, stream=None):
        E = self._points(E)
        if labels is None:
            labels = np.empty(E.shape[0], dtype=np.int32)
        _check(lib().igp_clusterer_predict(self.handle, _ptr(E), int(E.shape[0]), _ptr(labels), _stream(stream)))
        return labels

    def info(self, centroids=False, counts=False):
        """K, and the K x d centroids / K counts (numpy) if asked."""
        K = ctypes.c_int32()
        _check(lib().igp_clusterer_info(self.handle, ctypes.byref(K), None, None, None))
        C = np.empty((K.value, self.d), dtype=np.float32) if centroids else None
        n = np.empty(K.value, dtype=np.int64) if counts else None
        if K.value and (centroids or counts):
            _check(lib().igp_clusterer_info(self.handle, None, _ptr(C), _ptr(n), None))
        return K.value, C, n

    def free(self):
        if self.handle:
            lib().igp_clusterer_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """Owning wrapper of an igp_server: queued, memory-admitted, concurrent embed / append requests."""

    def __init__(self, slots=4, max_queue=0, reserve_bytes=1 << 30, device=-1, batch_rows=0):
        o = ServerOpts()
        lib().igp_server_opts_init(ctypes.byref(o))
        o.slots, o.max_queue, o.reserve_bytes, o.device = slots, max_queue, reserve_bytes, device
        o.batch_rows = batch_rows
        h = ctypes.c_void_p()
        _check(lib().igp_server_create(ctypes.byref(o), ctypes.byref(h)))
        self.handle = h.value
        self._outs = {}

    def submit(self, src, dst, N, tau, L, d, seed, kind="embed", graph_id=0, keep=False, out=None, **kw):
        """Queue a request (host int32 edge arrays, copied now); returns its ticket. The result lands in
        `out` (a new float32 (N - out_row_begin) x d array unless given), available from result() once done."""
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        if out is None:
            out = np.empty((max(int(N) - int(kw.get("out_row_begin", 0)), 0), d), dtype=np.float32)
        r = Request()
        r.kind = IGP_REQ_EMBED if kind == "embed" else IGP_REQ_APPEND
        r.keep = 1 if keep else 0
        r.graph_id = int(graph_id)
        r.src, r.dst, r.M, r.N = src.ctypes.data, dst.ctypes.data, src.size, int(N)
        r.tau, r.L, r.d, r.seed = float(tau), int(L), int(d), int(seed) & 0xFFFFFFFFFFFFFFFF
        r.opts = embed_opts(**kw)
        r.out = _ptr(out)
        t = ctypes.c_uint64()
        _check(lib().igp_submit(self.handle, ctypes.byref(r), ctypes.byref(t)))
        self._outs[t.value] = out
        return t.value

    def poll(self, ticket):
        st = ctypes.c_int32()
        lat = ctypes.c_double()
        code = lib().igp_poll(self.handle, ticket, ctypes.byref(st), ctypes.byref(lat))
        return REQ_STATES[st.value], lat.value, code

    def wait(self, ticket, timeout=-1.0):
        """Wait for a request; returns (state, latency_s); raises IgpError if it failed."""
        st = ctypes.c_int32()
        lat = ctypes.c_double()
        code = lib().igp_wait(self.handle, ticket, float(timeout), ctypes.byref(st), ctypes.byref(lat))
        if code not in (IGP_OK, IGP_E_NOTREADY, IGP_E_CANCELLED):
            raise IgpError(code, lib().igp_last_error().decode())
        return REQ_STATES[st.value], lat.value

    def result(self, ticket):
        return self._outs[ticket]

    def forget(self, ticket):
        """igp_server_forget: drop a finished request's record in the server and this wrapper's
        reference to its output, which is returned. Call it once a result has been read, so that
        a long-running server keeps nothing per past request. Raises IgpError (IGP_E_BUSY) while
        the request is queued or running."""
        _check(lib().igp_server_forget(self.handle, ticket))
        return self._outs.pop(ticket, None)

    def cancel(self, ticket):
        _check(lib().igp_cancel(self.handle, ticket))

    def release(self, graph_id):
        _check(lib().igp_server_release(self.handle, int(graph_id)))

    def stats(self):
        s = ServerStats()
        _check(lib().igp_server_get_stats(self.handle, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self.handle:
            lib().igp_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
