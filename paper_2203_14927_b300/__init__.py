"""GraphZeppelin hot path on B300: Python binding of the C ABI in include/gz.h.

Argument marshalling only -- every step (validation, partition by endpoint,
CubeSketch updates, Boruvka rounds) runs in the CUDA library ``libgz.so``
built from ``csrc/`` for sm_103a.  There is no CPU fallback: importing works
without a GPU, but creating a Graph needs the library and a CUDA device.

    g = Graph(V=1 << 13, seed=1)
    g.edge_update(u, v)            # torch CUDA tensors, or host numpy arrays
    labels, n_cc, stats = g.connected_components()
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgz.so")

GZ_OK, GZ_EINVAL, GZ_ENOMEM, GZ_ECUDA, GZ_ESKETCH_FAIL, GZ_ETIMEOUT, GZ_EBUSY = range(7)
KERNELS = {"batched": 0, "plain": 1}
COLS = 7


class GzError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"gz status {status}: {msg}")
        self.status = status


class SketchFailure(GzError):
    """The query finished but a CubeSketch failed; results are best effort."""


class Config(ctypes.Structure):
    _fields_ = [
        ("chunk_log2", ctypes.c_uint32),
        ("kernel", ctypes.c_uint32),
        ("smem_rows", ctypes.c_uint32),
        ("tile_records", ctypes.c_uint32),
        ("ctas_per_sm", ctypes.c_uint32),
        ("small_segment", ctypes.c_uint32),
        ("smem_mode", ctypes.c_uint32),
        ("no_graph", ctypes.c_uint32),
        ("device_sketch_mb", ctypes.c_uint32),
        ("no_pipeline", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32 * 2),
    ]


class Profile(ctypes.Structure):
    _fields_ = [
        ("batches", ctypes.c_uint64),
        ("updates", ctypes.c_uint64),
        ("partition_ms", ctypes.c_double),
        ("update_ms", ctypes.c_double),
        ("rows_flushed", ctypes.c_uint64),
        ("deep_updates", ctypes.c_uint64),
        ("kernel_launches", ctypes.c_uint64),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class KronParams(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_uint32),
        ("slice_log2", ctypes.c_uint32),
        ("k_feistel", ctypes.c_uint64 * 4),
        ("k_kron", ctypes.c_uint64),
        ("k_churn", ctypes.c_uint64),
        ("k_iso", ctypes.c_uint64),
        ("t_iso", ctypes.c_uint64),
        ("t_churn", ctypes.c_uint64),
    ]


class QueryStats(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_uint32),
        ("fails_last", ctypes.c_uint32),
        ("exhausted", ctypes.c_uint32),
        ("n_components", ctypes.c_uint32),
        ("fails_total", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
        ("ms", ctypes.c_float),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


_lib = None

# name -> (restype, argtypes); every symbol of include/gz.h
_SIGNATURES = {
    "gz_version": (ctypes.c_char_p, []),
    "gz_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "gz_geometry": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]),
    "gz_memory_bytes": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]),
    "gz_create": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p]),
    "gz_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "gz_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gz_edge_update": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                      ctypes.c_int]),
    "gz_edge_update_idx": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]),
    "gz_int_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p]),
    "gz_l0_geometry": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gz_l0_update": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                    ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    "gz_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "gz_reset": (ctypes.c_int, [ctypes.c_void_p]),
    "gz_connected_components": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p]),
    "gz_list_spanning_forest": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p]),
    "gz_enable_trace": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "gz_query_trace": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gz_export_sketch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int]),
    "gz_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_void_p]),
    "gz_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "gz_set_wait_limit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32]),
    "gz_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gz_gen_kron_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gz_gen_kron_num_chunks": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gz_gen_kron_chunk": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_uint64, ctypes.c_void_p]),
    "gz_gen_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "gz_server_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gz_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "gz_server_add_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "gz_server_submit_update": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32,
                                               ctypes.c_void_p]),
    "gz_server_submit_query": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                              ctypes.c_void_p]),
    "gz_server_close_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32]),
    "gz_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                      ctypes.c_int]),
    "gz_server_drain": (ctypes.c_int, [ctypes.c_void_p]),
    "gz_server_stats_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gz_server_set_budget": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "gz_server_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "gz_checkpoint_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gz_checkpoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "gz_restore": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p]),
    "gz_sketch_update_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                                ctypes.c_void_p, ctypes.c_void_p]),
}


def lib():
    """Load libgz.so (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing; build it with "
                               "`python -m paper_2203_14927_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def geometry(V: int) -> tuple[int, int]:
    K = ctypes.c_uint32()
    R = ctypes.c_uint32()
    if lib().gz_geometry(V, ctypes.byref(K), ctypes.byref(R)) != GZ_OK:
        raise ValueError(f"invalid V={V}")
    return K.value, R.value


def _config(kernel: str = "batched", chunk_log2: int = 0, smem_rows: int = 0, tile_records: int = 0,
            ctas_per_sm: int = 0, small_segment: int = 0, smem_mode: int = 0, no_graph: int = 0,
            device_sketch_mb: int = 0, no_pipeline: int = 0) -> Config:
    cfg = Config()
    cfg.chunk_log2 = chunk_log2
    cfg.kernel = KERNELS[kernel]
    cfg.smem_rows = smem_rows
    cfg.tile_records = tile_records
    cfg.ctas_per_sm = ctas_per_sm
    cfg.small_segment = small_segment
    cfg.smem_mode = smem_mode
    cfg.no_graph = no_graph
    cfg.device_sketch_mb = device_sketch_mb
    cfg.no_pipeline = no_pipeline
    return cfg


def memory_bytes(V: int, **cfg) -> int:
    """Device bytes a handle of V nodes allocates at creation (gz_memory_bytes)."""
    out = ctypes.c_size_t()
    st = lib().gz_memory_bytes(V, ctypes.byref(_config(**cfg)), ctypes.byref(out))
    if st != GZ_OK:
        raise GzError(st, "gz_memory_bytes failed")
    return out.value


def int_peak(kind: str = "mixed") -> float:
    """Measured integer thread-operations/s of the current device
    (gz_int_peak): "imad" (32-bit multiply-add), "lop3" (logic), "mixed" (the
    two interleaved), "clz" (leading-zero count) or "atom_shared" (32-bit
    shared-memory atomic XOR)."""
    out = ctypes.c_double()
    k = {"imad": 0, "lop3": 1, "mixed": 2, "clz": 3, "atom_shared": 4}[kind]
    st = lib().gz_int_peak(k, ctypes.byref(out))
    if st != GZ_OK:
        raise GzError(st, "gz_int_peak failed")
    return out.value


L0_CUBE, L0_STANDARD = 0, 1


def l0_geometry(n: int) -> tuple[int, int, int]:
    """(rows, bytes of a CubeSketch, bytes of a standard sketch) for length n."""
    r, bc, bs = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    st = lib().gz_l0_geometry(n, ctypes.byref(r), ctypes.byref(bc), ctypes.byref(bs))
    if st != GZ_OK:
        raise GzError(st, f"gz_l0_geometry(n={n}) failed")
    return r.value, bc.value, bs.value


def l0_update(kind: int, n: int, seed: int, x, buckets, delta=None, stream=None):
    """Apply x (torch int64 CUDA tensor, [sketches, m]) with optional +-1 deltas
    (int32, same shape) to `sketches` vector sketches in `buckets` (a CUDA
    tensor of sketches * bytes-per-sketch bytes); asynchronous."""
    sketches, m = x.shape
    s = _current_stream() if stream is None else stream
    st = lib().gz_l0_update(kind, n, seed & ((1 << 64) - 1), sketches, m, ctypes.c_void_p(x.data_ptr()),
                            ctypes.c_void_p(delta.data_ptr() if delta is not None else None),
                            ctypes.c_void_p(buckets.data_ptr()), ctypes.c_void_p(s))
    if st != GZ_OK:
        raise GzError(st, "gz_l0_update failed")


def _buffer(x, bits: int = 32):
    """(pointer, n, on_device, keepalive) of a 1-D unsigned/signed integer
    array of the given width (32 for vertex ids, 64 for packed indices)."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        ok = (torch.int32, torch.uint32) if bits == 32 else (torch.int64, torch.uint64)
        if x.dtype not in ok:
            raise TypeError(f"update tensors must be int{bits} or uint{bits}")
        x = x.contiguous().reshape(-1)
        return x.data_ptr(), x.numel(), 1 if x.is_cuda else 0, x
    a = np.asarray(x)
    signed, unsigned = (np.int32, np.uint32) if bits == 32 else (np.int64, np.uint64)
    if a.dtype == signed and a.flags["C_CONTIGUOUS"]:
        a = a.view(unsigned)  # same bytes, no copy (keeps pinned memory pinned)
    a = np.ascontiguousarray(a, dtype=unsigned).reshape(-1)
    return a.ctypes.data, a.size, 0, a


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover
        pass
    return 0


class Graph:
    """Node sketches of one dynamic graph resident on the current CUDA device."""

    def __init__(self, V: int, seed: int = 0, *, kernel: str = "batched", chunk_log2: int = 0,
                 smem_rows: int = 0, tile_records: int = 0, ctas_per_sm: int = 0,
                 small_segment: int = 0, smem_mode: int = 0, no_graph: int = 0, device_sketch_mb: int = 0,
                 no_pipeline: int = 0, stream=None):
        cfg = _config(kernel=kernel, chunk_log2=chunk_log2, smem_rows=smem_rows, tile_records=tile_records,
                      ctas_per_sm=ctas_per_sm, small_segment=small_segment, smem_mode=smem_mode,
                      no_graph=no_graph, device_sketch_mb=device_sketch_mb, no_pipeline=no_pipeline)
        self._h = ctypes.c_void_p()
        s = _current_stream() if stream is None else stream
        st = lib().gz_create(V, seed & ((1 << 64) - 1), ctypes.byref(cfg), ctypes.c_void_p(s),
                             ctypes.byref(self._h))
        if st != GZ_OK:
            raise GzError(st, f"gz_create(V={V}) failed: {lib().gz_last_error(None).decode()}")
        self.V = V
        self.seed = seed
        self.K, self.R = geometry(V)

    # -- plumbing --------------------------------------------------------------
    def _check(self, st: int, what: str):
        if st == GZ_OK:
            return
        msg = lib().gz_last_error(self._h).decode()
        if st == GZ_ESKETCH_FAIL:
            raise SketchFailure(st, f"{what}: {msg}")
        raise GzError(st, f"{what}: {msg}")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().gz_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream: int):
        self._check(lib().gz_set_stream(self._h, ctypes.c_void_p(stream)), "gz_set_stream")

    # -- ingestion ---------------------------------------------------------------
    def edge_update(self, u, v):
        pu, nu, du, ku = _buffer(u)
        pv, nv, dv, kv = _buffer(v)
        if nu != nv or du != dv:
            raise ValueError("u and v must have equal length and live on the same side")
        self._check(lib().gz_edge_update(self._h, ctypes.c_void_p(pu), ctypes.c_void_p(pv), nu, du),
                    "gz_edge_update")
        return ku, kv

    def edge_update_idx(self, idx):
        """Updates as packed indices min(u,v)*V + max(u,v) (int64/uint64)."""
        p, n, d, k = _buffer(idx, 64)
        self._check(lib().gz_edge_update_idx(self._h, ctypes.c_void_p(p), n, d), "gz_edge_update_idx")
        return k

    def sync(self):
        self._check(lib().gz_sync(self._h), "gz_sync")

    def reset(self):
        self._check(lib().gz_reset(self._h), "gz_reset")

    # -- queries -------------------------------------------------------------------
    def connected_components(self, raise_on_failure: bool = False):
        labels = np.zeros(self.V, np.uint32)
        ncc = ctypes.c_uint32()
        st = QueryStats()
        rc = lib().gz_connected_components(self._h, labels.ctypes.data_as(ctypes.c_void_p),
                                           ctypes.byref(ncc), ctypes.byref(st))
        if rc != GZ_ESKETCH_FAIL or raise_on_failure:
            self._check(rc, "gz_connected_components")
        d = st.as_dict()
        d["status"] = rc
        return labels, ncc.value, d

    def list_spanning_forest(self, raise_on_failure: bool = False):
        uv = np.zeros(2 * max(self.V - 1, 1), np.uint32)
        n = ctypes.c_size_t()
        labels = np.zeros(self.V, np.uint32)
        st = QueryStats()
        rc = lib().gz_list_spanning_forest(self._h, uv.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n),
                                           labels.ctypes.data_as(ctypes.c_void_p), ctypes.byref(st))
        if rc != GZ_ESKETCH_FAIL or raise_on_failure:
            self._check(rc, "gz_list_spanning_forest")
        d = st.as_dict()
        d["status"] = rc
        return uv[: 2 * n.value].reshape(-1, 2).copy(), labels, d

    def enable_trace(self, on: bool = True):
        self._check(lib().gz_enable_trace(self._h, 1 if on else 0), "gz_enable_trace")

    def query_trace(self) -> np.ndarray:
        out = np.zeros(self.K * self.V, np.int64)
        self._check(lib().gz_query_trace(self._h, out.ctypes.data_as(ctypes.c_void_p)), "gz_query_trace")
        return out.reshape(self.K, self.V)

    def export_sketch(self, lo: int = 0, hi: int | None = None):
        """Nested-form sketches of nodes [lo, hi): alpha/gamma [node][k][j][row]."""
        hi = self.V if hi is None else hi
        a = np.zeros((hi - lo, self.K, COLS, self.R), np.uint64)
        g = np.zeros((hi - lo, self.K, COLS, self.R), np.uint32)
        self._check(lib().gz_export_sketch(self._h, lo, hi, a.ctypes.data_as(ctypes.c_void_p),
                                           g.ctypes.data_as(ctypes.c_void_p), 0), "gz_export_sketch")
        return a, g

    def checkpoint(self) -> np.ndarray:
        """The handle's whole state as bytes (header + node sketches)."""
        n = ctypes.c_size_t()
        self._check(lib().gz_checkpoint_bytes(self._h, ctypes.byref(n)), "gz_checkpoint_bytes")
        buf = np.empty(n.value, np.uint8)
        self._check(lib().gz_checkpoint(self._h, buf.ctypes.data_as(ctypes.c_void_p), n.value), "gz_checkpoint")
        return buf

    @classmethod
    def restore(cls, buf, stream=None, **cfg) -> "Graph":
        """A new Graph holding exactly the checkpointed state."""
        buf = np.ascontiguousarray(buf, np.uint8)
        c = Config()
        for k, val in cfg.items():
            setattr(c, k, KERNELS[val] if k == "kernel" else val)
        h = ctypes.c_void_p()
        s = _current_stream() if stream is None else stream
        st = lib().gz_restore(buf.ctypes.data_as(ctypes.c_void_p), buf.size, ctypes.byref(c), ctypes.c_void_p(s),
                              ctypes.byref(h))
        if st != GZ_OK:
            raise GzError(st, "gz_restore failed")
        g = cls.__new__(cls)
        g._h = h
        info = g.info()
        g.V = info["V"]
        g.K, g.R = info["K"], info["R"]
        g.seed = int(np.frombuffer(buf[24:32].tobytes(), np.uint64)[0])
        return g

    def set_wait_limit(self, polls: int, suspend_ns: int = 0):
        """Bound the update kernel's waits (polls = 0: the defaults)."""
        self._check(lib().gz_set_wait_limit(self._h, polls, suspend_ns), "gz_set_wait_limit")

    def profile_enable(self, on: bool = True):
        self._check(lib().gz_profile_enable(self._h, 1 if on else 0), "gz_profile_enable")

    def profile_read(self) -> dict:
        p = Profile()
        self._check(lib().gz_profile_read(self._h, ctypes.byref(p)), "gz_profile_read")
        return p.as_dict()

    def info(self) -> dict:
        V, K, R = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        nb = ctypes.c_size_t()
        ptr = ctypes.c_void_p()
        self._check(lib().gz_info(self._h, ctypes.byref(V), ctypes.byref(K), ctypes.byref(R),
                                  ctypes.byref(nb), ctypes.byref(ptr)), "gz_info")
        return {"V": V.value, "K": K.value, "R": R.value, "node_bytes": nb.value, "sketch_ptr": ptr.value}


class DeviceKronStream:
    """Device generator of the chunks of a streams.KronSpec (same updates as
    KronSpec.chunk on the host)."""

    def __init__(self, spec, stream=None):
        d = spec.device_params()
        p = KronParams()
        p.L = d["L"]
        p.slice_log2 = d["slice_log2"]
        for i, k in enumerate(d["k_feistel"]):
            p.k_feistel[i] = k
        p.k_kron, p.k_churn, p.k_iso = d["k_kron"], d["k_churn"], d["k_iso"]
        p.t_iso, p.t_churn = d["t_iso"], d["t_churn"]
        self._table = np.ascontiguousarray(d["table"], np.uint64)
        self._g = ctypes.c_void_p()
        s = _current_stream() if stream is None else stream
        st = lib().gz_gen_kron_create(ctypes.byref(p), self._table.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.c_void_p(s), ctypes.byref(self._g))
        if st != GZ_OK:
            raise GzError(st, "gz_gen_kron_create failed")
        n = ctypes.c_uint64()
        lib().gz_gen_kron_num_chunks(self._g, ctypes.byref(n))
        self.n_chunks = n.value
        self.spec = spec

    def chunk_into(self, c: int, u_ptr: int, v_ptr: int, capacity: int) -> int:
        """Write chunk c to device pointers; returns its length."""
        n = ctypes.c_uint64()
        st = lib().gz_gen_kron_chunk(self._g, c, ctypes.c_void_p(u_ptr), ctypes.c_void_p(v_ptr), capacity,
                                     ctypes.byref(n))
        if st != GZ_OK:
            raise GzError(st, f"gz_gen_kron_chunk({c}) failed")
        return n.value

    def chunk(self, c: int):
        """Chunk c as a pair of int32 CUDA tensors (bit patterns of uint32 ids)."""
        import torch
        cap = int(self.spec.slice_len * 2 + 16)
        u = torch.empty(cap, dtype=torch.int32, device="cuda")
        v = torch.empty(cap, dtype=torch.int32, device="cuda")
        n = self.chunk_into(c, u.data_ptr(), v.data_ptr(), cap)
        return u[:n], v[:n]

    def close(self):
        if getattr(self, "_g", None) and self._g.value:
            lib().gz_gen_destroy(self._g)
            self._g = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("slots", ctypes.c_uint32), ("max_batch", ctypes.c_uint32),
                ("host_pool_mb", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 5)]


class Completion(ctypes.Structure):
    _fields_ = [("req_id", ctypes.c_uint64), ("graph", ctypes.c_uint32), ("kind", ctypes.c_uint32),
                ("status", ctypes.c_int32), ("n_components", ctypes.c_uint32), ("n_updates", ctypes.c_uint64),
                ("submit_ms", ctypes.c_double), ("start_ms", ctypes.c_double), ("done_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("resident_bytes", ctypes.c_uint64), ("peak_resident_bytes", ctypes.c_uint64),
                ("budget_bytes", ctypes.c_uint64), ("graphs", ctypes.c_uint32),
                ("resident_graphs", ctypes.c_uint32), ("waiting_graphs", ctypes.c_uint32),
                ("pending_requests", ctypes.c_uint32), ("completed_requests", ctypes.c_uint64),
                ("evictions", ctypes.c_uint64), ("evicted_graphs", ctypes.c_uint32), ("pinned_chunks", ctypes.c_uint32),
                ("evict_ms", ctypes.c_double), ("restore_ms", ctypes.c_double)]


class Server:
    """Many graphs resident on the current device (gz_server_* in include/gz.h):
    admission by an HBM budget, `slots` concurrent workers (streams)."""

    def __init__(self, hbm_budget: int = 0, slots: int = 0, max_batch: int = 0, host_pool_mb: int = 0):
        cfg = ServerConfig()
        cfg.hbm_budget, cfg.slots, cfg.max_batch, cfg.host_pool_mb = hbm_budget, slots, max_batch, host_pool_mb
        self._s = ctypes.c_void_p()
        st = lib().gz_server_create(ctypes.byref(cfg), ctypes.byref(self._s))
        if st != GZ_OK:
            raise GzError(st, "gz_server_create failed")
        self._labels = {}
        self._lent = {}
        self._V = {}

    def add_graph(self, V: int, seed: int = 0, **cfg) -> int:
        c = Config()
        for k, val in cfg.items():
            setattr(c, k, KERNELS[val] if k == "kernel" else val)
        gid = ctypes.c_uint32()
        st = lib().gz_server_add_graph(self._s, V, seed & ((1 << 64) - 1), ctypes.byref(c), ctypes.byref(gid))
        if st != GZ_OK:
            raise GzError(st, f"gz_server_add_graph(V={V}) failed")
        self._V[gid.value] = V
        return gid.value

    def submit_update(self, graph: int, u, v, copy: bool = True) -> int:
        """Queue an update batch.  copy=False lends the arrays to the server
        (kept alive here until the completion is polled)."""
        u = np.asarray(u)
        v = np.asarray(v)
        if u.dtype == np.int32:
            u = u.view(np.uint32)
        if v.dtype == np.int32:
            v = v.view(np.uint32)
        u = np.ascontiguousarray(u, np.uint32)
        v = np.ascontiguousarray(v, np.uint32)
        rid = ctypes.c_uint64()
        st = lib().gz_server_submit_update(self._s, graph, u.ctypes.data_as(ctypes.c_void_p),
                                           v.ctypes.data_as(ctypes.c_void_p), len(u),
                                           0 if copy else 1, ctypes.byref(rid))
        if st != GZ_OK:
            raise GzError(st, "gz_server_submit_update failed")
        if not copy:
            self._lent[rid.value] = (u, v)
        return rid.value

    def submit_query(self, graph: int) -> int:
        labels = np.zeros(self._V[graph], np.uint32)
        rid = ctypes.c_uint64()
        st = lib().gz_server_submit_query(self._s, graph, labels.ctypes.data_as(ctypes.c_void_p),
                                          ctypes.byref(rid))
        if st != GZ_OK:
            raise GzError(st, "gz_server_submit_query failed")
        self._labels[rid.value] = labels
        return rid.value

    def close_graph(self, graph: int):
        lib().gz_server_close_graph(self._s, graph)

    def poll(self, max_n: int = 4096, wait_ms: int = 0) -> list:
        buf = (Completion * max_n)()
        n = ctypes.c_size_t()
        lib().gz_server_poll(self._s, buf, max_n, ctypes.byref(n), wait_ms)
        out = []
        for i in range(n.value):
            c = buf[i]
            d = {f: getattr(c, f) for f, _ in Completion._fields_}
            if c.kind == 1:
                d["labels"] = self._labels.pop(c.req_id, None)
            else:
                self._lent.pop(c.req_id, None)
            out.append(d)
        return out

    def drain(self):
        lib().gz_server_drain(self._s)

    def last_error(self) -> str:
        return lib().gz_server_last_error(self._s).decode()

    def set_budget(self, hbm_budget: int):
        st = lib().gz_server_set_budget(self._s, int(hbm_budget))
        if st != GZ_OK:
            raise GzError(st, "gz_server_set_budget failed")

    def stats(self) -> dict:
        st = ServerStats()
        lib().gz_server_stats_read(self._s, ctypes.byref(st))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_s", None) and self._s.value:
            lib().gz_server_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
