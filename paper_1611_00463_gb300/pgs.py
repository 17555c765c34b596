"""Python binding of libpgs.so: the C ABI of include/pgs.h, argument marshalling only.

Every step of the sort runs in the library's CUDA kernels; PyTorch only provides
device memory (the tensors and the workspace) and the stream.  There is no CPU
fallback: if the library is missing or the tensors are not on a CUDA device the
calls raise.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpgs.so")

PGS_U32, PGS_U64, PGS_F32 = 0, 1, 2
PGS_OK, PGS_ERR_INVALID, PGS_ERR_WORKSPACE, PGS_ERR_CUDA, PGS_ERR_TIMEOUT, PGS_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5
INVESTIGATOR = {"rank": 0, "equal": 1, "off": 2, "local": 3}
EXCHANGE = {"auto": 0, "scatter": 1, "fused": 2}
SPLITTERS = {"sampled": 0, "learned": 1}
COPY_BACK = {"auto": 0, "end": 1, "groups": 2}
GRAPH_CACHE = {"auto": 0, "off": 1}
FAULT_INJECT = {"off": 0, "wait_timeout": 1}     # testing only (pgs_config.fault_inject)
DTYPES = {"u32": PGS_U32, "u64": PGS_U64, "f32": PGS_F32}
KEY_TORCH = {"u32": torch.int32, "u64": torch.int64, "f32": torch.int32}
MLP_FLOATS = 1 * 32 + 32 + 32 * 32 + 32 + 32 * 1 + 1
MLP_WORDS = MLP_FLOATS + 4


class pgs_config(ctypes.Structure):
    _fields_ = [
        ("dtype", ctypes.c_int32),
        ("samples_per_run", ctypes.c_uint32),
        ("eps", ctypes.c_float),
        ("guaranteed", ctypes.c_int32),
        ("investigator", ctypes.c_int32),
        ("exchange", ctypes.c_int32),
        ("splitter_mode", ctypes.c_int32),
        ("tile_variant", ctypes.c_int32),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_uint64),
        ("bucket_bounds", ctypes.c_void_p),
        ("cuts", ctypes.c_void_p),
        ("splitters", ctypes.c_void_p),
        ("stats", ctypes.c_void_p),
        ("spin_limit", ctypes.c_uint64),
        ("timer", ctypes.c_void_p),
        ("model", ctypes.c_void_p),
        ("model_out", ctypes.c_void_p),
        ("merge_ways", ctypes.c_int32),
        ("copy_back", ctypes.c_int32),
        ("graph_cache", ctypes.c_int32),
        ("fault_inject", ctypes.c_int32),
    ]


class pgs_stats(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint64),
        ("P", ctypes.c_uint32),
        ("samples_per_run", ctypes.c_uint32),
        ("max_bucket", ctypes.c_uint64),
        ("min_bucket", ctypes.c_uint64),
        ("splitter_mode", ctypes.c_uint32),
        ("fallback", ctypes.c_uint32),
        ("error", ctypes.c_uint32),
        ("passes", ctypes.c_uint32),
        ("launches", ctypes.c_uint32),
        ("max_over_mean", ctypes.c_float),
        ("learned_over_mean", ctypes.c_float),
        ("reserved", ctypes.c_uint32),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = {
    "pgs_workspace_bytes": (ctypes.c_size_t, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p]),
    "pgs_sort": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                ctypes.c_void_p, ctypes.c_void_p]),
    "pgs_sort_copy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]),
    "pgs_sort_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "pgs_host_workspace_bytes": (ctypes.c_size_t, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p]),
    "pgs_sort_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]),
    "pgs_search": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p]),
    "pgs_search_workspace_bytes": (ctypes.c_size_t, [ctypes.c_uint64, ctypes.c_void_p]),
    "pgs_provenance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pgs_fit_workspace_bytes": (ctypes.c_size_t, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p]),
    "pgs_fit_splitters": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pgs_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pgs_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "pgs_version": (ctypes.c_char_p, []),
    "pgs_last_error": (ctypes.c_char_p, []),
    "pgs_timer_create": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_void_p]),
    "pgs_timer_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "pgs_timer_reset": (ctypes.c_int, [ctypes.c_void_p]),
    "pgs_timer_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "pgs_kernel_name": (ctypes.c_char_p, [ctypes.c_uint32]),
    "pgs_batch_auto_partitions": (ctypes.c_uint32, [ctypes.c_uint64]),
    "pgs_batch_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "pgs_batch_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "pgs_batch_upload": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
    "pgs_sort_batched": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "pgs_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "pgs_sort_batched_copy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pgs_samples_per_run": (ctypes.c_uint64, [ctypes.c_uint32, ctypes.c_void_p]),
    "pgs_rank_samples": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "pgs_rank_counts": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint32,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pgs_rank_cuts_workspace_bytes": (ctypes.c_size_t, [ctypes.c_uint32, ctypes.c_void_p]),
    "pgs_rank_cuts": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pgs_merge_workspace_bytes": (ctypes.c_size_t, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p]),
    "pgs_merge_lists": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pgs_batch_tune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
}
TILE_VARIANTS = 4

KERNELS = ["block_sort", "merge", "partition", "pairs", "scan", "sample", "splitters", "cut_search",
           "investigator", "offsets", "scatter", "stats", "merge4"]


class pgs_launch_record(ctypes.Structure):
    _fields_ = [
        ("kernel", ctypes.c_uint32),
        ("step", ctypes.c_uint32),
        ("bytes", ctypes.c_uint64),
        ("ms", ctypes.c_float),
        ("reserved", ctypes.c_uint32),
    ]

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libpgs.so (built by paper_1611_00463_gb300.build) and declare its exports."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1611_00463_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class PgsError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        detail = pgs_last_error() if status == PGS_ERR_CUDA else ""
        super().__init__(f"{what}: {pgs_strerror(status)} ({status}) {detail}".rstrip())


def _check(status: int, what: str) -> None:
    if status != PGS_OK:
        raise PgsError(status, what)


def pgs_strerror(status: int) -> str:
    return load().pgs_strerror(status).decode()


def pgs_version() -> str:
    return load().pgs_version().decode()


def pgs_last_error() -> str:
    return load().pgs_last_error().decode()


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensors passed to the CUDA sort must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return t.data_ptr()


def _host_ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    if t.is_cuda or not t.is_contiguous():
        raise ValueError("pgs_sort_host takes contiguous host tensors")
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


class Timer:
    """Owner of a pgs_timer (the launch timer of the C ABI)."""

    def __init__(self, capacity: int = 4096):
        h = ctypes.c_void_p()
        _check(load().pgs_timer_create(capacity, ctypes.byref(h)), "pgs_timer_create")
        self.handle = h.value
        self.capacity = capacity

    def reset(self) -> None:
        _check(load().pgs_timer_reset(self.handle), "pgs_timer_reset")

    def read(self) -> tuple[list[dict], int]:
        """Wait for the recorded launches; returns ([{kernel, step, bytes, ms}], dropped)."""
        buf = (pgs_launch_record * self.capacity)()
        cnt, drop = ctypes.c_uint32(), ctypes.c_uint32()
        _check(load().pgs_timer_read(self.handle, buf, self.capacity, ctypes.byref(cnt), ctypes.byref(drop)),
               "pgs_timer_read")
        out = [{"kernel": KERNELS[r.kernel], "step": r.step, "bytes": r.bytes, "ms": r.ms}
               for r in buf[:cnt.value]]
        return out, drop.value

    def close(self) -> None:
        if self.handle:
            load().pgs_timer_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_config(dtype: str = "u32", samples_per_run: int = 0, eps: float = 0.0, guaranteed: bool = False,
                investigator: str = "rank", exchange: str = "auto", splitters: str = "sampled",
                workspace: torch.Tensor | None = None, bucket_bounds: torch.Tensor | None = None,
                cuts: torch.Tensor | None = None, splitters_out: torch.Tensor | None = None,
                stats: torch.Tensor | None = None, timer: Timer | None = None,
                model: torch.Tensor | None = None, model_out: torch.Tensor | None = None,
                tile_variant: int = 0, merge_ways: int = 0, copy_back: str = "auto",
                graph_cache: str = "auto", spin_limit: int = 0, fault_inject: str = "off") -> pgs_config:
    """The options of a call.  The struct holds raw device addresses, so it
    also keeps a reference to every tensor (and the timer) it points to: they
    live as long as the config does, and `make_config(workspace=workspace(...))`
    cannot leave the library writing into memory the allocator has handed on."""
    c = pgs_config()
    c._keep = tuple(x for x in (workspace, bucket_bounds, cuts, splitters_out, stats, timer, model, model_out)
                    if x is not None)
    c.dtype = DTYPES[dtype]
    c.samples_per_run = samples_per_run
    c.eps = eps
    c.guaranteed = int(guaranteed)
    c.investigator = INVESTIGATOR[investigator]
    c.exchange = EXCHANGE[exchange]
    c.splitter_mode = SPLITTERS[splitters]
    if workspace is not None:
        c.workspace = _ptr(workspace)
        c.workspace_bytes = workspace.numel() * workspace.element_size()
    c.bucket_bounds = _ptr(bucket_bounds)
    c.cuts = _ptr(cuts)
    c.splitters = _ptr(splitters_out)
    c.stats = _ptr(stats)
    c.timer = timer.handle if timer is not None else None
    c.model = _ptr(model)
    c.model_out = _ptr(model_out)
    c.tile_variant = tile_variant
    c.merge_ways = merge_ways
    c.copy_back = COPY_BACK[copy_back]
    c.graph_cache = GRAPH_CACHE[graph_cache]
    c.spin_limit = spin_limit
    c.fault_inject = FAULT_INJECT[fault_inject]
    return c


def pgs_workspace_bytes(n: int, P: int, cfg: pgs_config | None = None) -> int:
    return load().pgs_workspace_bytes(n, P, ctypes.byref(cfg) if cfg is not None else None)


def workspace(n: int, P: int, cfg: pgs_config | None = None, device=None) -> torch.Tensor:
    """A device workspace tensor (256-byte aligned by the caching allocator)."""
    nbytes = pgs_workspace_bytes(n, P, cfg)
    if nbytes == 0:
        raise PgsError(PGS_ERR_INVALID, "pgs_workspace_bytes")
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def pgs_sort_copy(keys_in: torch.Tensor, vals_in: torch.Tensor | None, keys_out: torch.Tensor,
                  vals_out: torch.Tensor | None, P: int, cfg: pgs_config, stream=None) -> None:
    n = keys_in.numel()
    if keys_out.numel() != n or (vals_in is not None and (vals_in.numel() != n or vals_out.numel() != n)):
        raise ValueError("length mismatch")
    _check(load().pgs_sort_copy(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out), n, P,
                                _stream(stream), ctypes.byref(cfg)), "pgs_sort_copy")


def pgs_sort(keys: torch.Tensor, vals: torch.Tensor | None, P: int, cfg: pgs_config, stream=None) -> None:
    n = keys.numel()
    if vals is not None and vals.numel() != n:
        raise ValueError("length mismatch")
    _check(load().pgs_sort(_ptr(keys), _ptr(vals), n, P, _stream(stream), ctypes.byref(cfg)), "pgs_sort")


def pgs_host_workspace_bytes(n: int, P: int, cfg: pgs_config | None = None) -> int:
    return load().pgs_host_workspace_bytes(n, P, ctypes.byref(cfg) if cfg is not None else None)


def pgs_sort_host(keys_in: torch.Tensor, vals_in: torch.Tensor | None, keys_out: torch.Tensor,
                  vals_out: torch.Tensor | None, P: int, cfg: pgs_config, stream=None) -> None:
    """Host tensors in and out (pinned for full copy rate); the copies run
    inside the library, overlapped with steps 1 and 6.  The call waits for
    steps 1-5; the rest is asynchronous on `stream`."""
    n = keys_in.numel()
    if keys_out.numel() != n or (vals_in is not None and (vals_in.numel() != n or vals_out.numel() != n)):
        raise ValueError("length mismatch")
    _check(load().pgs_sort_host(_host_ptr(keys_in), _host_ptr(vals_in), _host_ptr(keys_out), _host_ptr(vals_out),
                                n, P, _stream(stream), ctypes.byref(cfg)), "pgs_sort_host")


def pgs_search_workspace_bytes(n: int, dtype: str = "u32") -> int:
    cfg = make_config(dtype=dtype)
    return load().pgs_search_workspace_bytes(n, ctypes.byref(cfg))


def pgs_search(keys: torch.Tensor, queries: torch.Tensor, pos_out: torch.Tensor, side: str = "left",
               dtype: str = "u32", bucket_bounds: torch.Tensor | None = None, bucket_out: torch.Tensor | None = None,
               workspace: torch.Tensor | None = None, stream=None) -> None:
    """Lower ("left") or upper ("right") bound of every query in sorted keys;
    with the sort's bucket bounds, also the bucket holding each position.  A
    workspace of pgs_search_workspace_bytes(n) bytes enables the indexed search."""
    if side not in ("left", "right"):
        raise ValueError(side)
    P = bucket_bounds.numel() - 1 if bucket_bounds is not None else 0
    if pos_out.numel() != queries.numel() or (bucket_out is not None and bucket_out.numel() != queries.numel()):
        raise ValueError("length mismatch")
    cfg = make_config(dtype=dtype, workspace=workspace)
    _check(load().pgs_search(_ptr(keys) if keys.numel() else None, keys.numel(), _ptr(queries), queries.numel(),
                             1 if side == "right" else 0, _ptr(bucket_bounds), P, _ptr(pos_out), _ptr(bucket_out),
                             _stream(stream), ctypes.byref(cfg)), "pgs_search")


def pgs_provenance(vals: torch.Tensor, n: int, P: int, run_out: torch.Tensor | None, index_out: torch.Tensor | None,
                   stream=None) -> None:
    """Previous processor (run) and index of entries whose payload is their input position."""
    _check(load().pgs_provenance(_ptr(vals), vals.numel(), n, P, _ptr(run_out), _ptr(index_out), _stream(stream)),
           "pgs_provenance")


STATIC_MAX_KEYS = 1 << 16
STATIC_MAX_P = 64
STATIC_SCRATCH_BYTES = 8 << 20


def pgs_sort_static(keys: torch.Tensor, vals: torch.Tensor | None, P: int, cfg: pgs_config | None = None,
                    stream=None) -> None:
    """In-place sort that uses the library's own static scratch (no workspace,
    no allocation); n <= STATIC_MAX_KEYS, P <= STATIC_MAX_P."""
    n = keys.numel()
    if vals is not None and vals.numel() != n:
        raise ValueError("length mismatch")
    cfg = cfg if cfg is not None else pgs_config()
    _check(load().pgs_sort_static(_ptr(keys), _ptr(vals), n, P, _stream(stream), ctypes.byref(cfg)),
           "pgs_sort_static")


def pgs_batch_auto_partitions(n: int) -> int:
    return load().pgs_batch_auto_partitions(n)


class Batch:
    """A batch of independent sort instances (pgs_batch_create / upload / sort).

    offsets: host sequence of num+1 key offsets; P: host sequence of num
    partition counts, or None for the automatic rule."""

    def __init__(self, offsets, P=None, dtype: str = "u32", with_vals: bool = True, device=None, **opts):
        import numpy as np
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
        self.num = len(off) - 1
        self.n = int(off[-1])
        pv = None if P is None else np.ascontiguousarray(np.asarray(P, dtype=np.uint32))
        self.dtype = dtype
        self.opts = opts
        cfg = make_config(dtype=dtype, **opts)
        h = ctypes.c_void_p()
        _check(load().pgs_batch_create(off.ctypes.data, self.num, pv.ctypes.data if pv is not None else None,
                                       int(with_vals), ctypes.byref(cfg), ctypes.byref(h)), "pgs_batch_create")
        self.handle = h.value
        nbytes = load().pgs_batch_workspace_bytes(self.handle)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")
        _check(load().pgs_batch_upload(self.handle, self.workspace.data_ptr(), nbytes,
                                       _stream(None)), "pgs_batch_upload")

    def config(self, stats: torch.Tensor | None = None, timer: "Timer | None" = None) -> pgs_config:
        return make_config(dtype=self.dtype, workspace=self.workspace, stats=stats, timer=timer, **self.opts)

    def sort(self, keys: torch.Tensor, vals: torch.Tensor | None, stream=None, cfg: pgs_config | None = None):
        """Sort every instance of keys (and vals) in place."""
        if keys.numel() != self.n or (vals is not None and vals.numel() != self.n):
            raise ValueError("length mismatch")
        cfg = cfg if cfg is not None else self.config()
        _check(load().pgs_sort_batched(self.handle, _ptr(keys), _ptr(vals), _stream(stream), ctypes.byref(cfg)),
               "pgs_sort_batched")

    def sort_copy(self, keys_in: torch.Tensor, vals_in: torch.Tensor | None, keys_out: torch.Tensor,
                  vals_out: torch.Tensor | None, stream=None, cfg: pgs_config | None = None):
        """Sort every instance of keys_in (and vals_in) into keys_out (and vals_out)."""
        for t in (keys_in, keys_out):
            if t.numel() != self.n:
                raise ValueError("length mismatch")
        cfg = cfg if cfg is not None else self.config()
        _check(load().pgs_sort_batched_copy(self.handle, _ptr(keys_in), _ptr(vals_in), _ptr(keys_out),
                                            _ptr(vals_out), _stream(stream), ctypes.byref(cfg)),
               "pgs_sort_batched_copy")

    def tune(self, scratch_keys: torch.Tensor, scratch_vals: torch.Tensor | None, stream=None):
        """Time every merge tile shape on pseudo-random keys in the scratch
        buffers and keep the fastest; returns (chosen, [ms per shape])."""
        chosen = ctypes.c_uint32()
        ms = (ctypes.c_float * TILE_VARIANTS)()
        cfg = self.config()
        _check(load().pgs_batch_tune(self.handle, _ptr(scratch_keys), _ptr(scratch_vals), _stream(stream),
                                     ctypes.byref(cfg), ctypes.byref(chosen), ms), "pgs_batch_tune")
        return chosen.value, list(ms)

    def close(self):
        if self.handle:
            load().pgs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Rank steps of the sharded sort (argument marshalling; the driver that runs
# them with collectives is paper_1611_00463_gb300.sharded).
# ---------------------------------------------------------------------------

def pgs_samples_per_run(P: int, cfg: pgs_config | None = None) -> int:
    return load().pgs_samples_per_run(P, ctypes.byref(cfg) if cfg is not None else None)


def pgs_rank_samples(sorted_keys: torch.Tensor, s: int, samples_out: torch.Tensor, cfg: pgs_config,
                     stream=None) -> None:
    _check(load().pgs_rank_samples(_ptr(sorted_keys), sorted_keys.numel(), s, _ptr(samples_out), _stream(stream),
                                   ctypes.byref(cfg)), "pgs_rank_samples")


def pgs_rank_counts(sorted_keys: torch.Tensor, splitters: torch.Tensor, G: int, counts_out: torch.Tensor,
                    cfg: pgs_config, stream=None) -> None:
    _check(load().pgs_rank_counts(_ptr(sorted_keys) if sorted_keys.numel() else None, sorted_keys.numel(),
                                  _ptr(splitters), G, _ptr(counts_out), _stream(stream), ctypes.byref(cfg)),
           "pgs_rank_counts")


def pgs_rank_cuts_workspace_bytes(G: int, cfg: pgs_config | None = None) -> int:
    return load().pgs_rank_cuts_workspace_bytes(G, ctypes.byref(cfg) if cfg is not None else None)


def pgs_rank_cuts(counts_all: torch.Tensor, shard_sizes, splitters: torch.Tensor, cut_out: torch.Tensor,
                  bounds_out: torch.Tensor, cfg: pgs_config, stream=None) -> None:
    """shard_sizes: host sequence of G sizes."""
    import numpy as np
    sizes = np.ascontiguousarray(np.asarray(shard_sizes, dtype=np.uint64))
    G = len(sizes)
    _check(load().pgs_rank_cuts(_ptr(counts_all) if G > 1 else None, sizes.ctypes.data, G,
                                _ptr(splitters) if G > 1 else None, _ptr(cut_out), _ptr(bounds_out), _stream(stream),
                                ctypes.byref(cfg)), "pgs_rank_cuts")


def pgs_merge_workspace_bytes(n: int, k: int, cfg: pgs_config | None = None) -> int:
    return load().pgs_merge_workspace_bytes(n, k, ctypes.byref(cfg) if cfg is not None else None)


def pgs_merge_lists(keys_in: torch.Tensor, vals_in: torch.Tensor | None, offsets, keys_out: torch.Tensor,
                    vals_out: torch.Tensor | None, cfg: pgs_config, stream=None) -> None:
    """offsets: host sequence of k+1 list offsets into keys_in."""
    import numpy as np
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
    k = len(off) - 1
    n = int(off[-1]) if k >= 0 else 0
    if keys_in.numel() < n or keys_out.numel() < n:
        raise ValueError("length mismatch")
    _check(load().pgs_merge_lists(_ptr(keys_in) if n else None, _ptr(vals_in) if n else None, off.ctypes.data, k,
                                  _ptr(keys_out) if n else None, _ptr(vals_out) if n else None, _stream(stream),
                                  ctypes.byref(cfg)), "pgs_merge_lists")


def pgs_fit_workspace_bytes(m: int, P: int, cfg: pgs_config | None = None) -> int:
    return load().pgs_fit_workspace_bytes(m, P, ctypes.byref(cfg) if cfg is not None else None)


def pgs_fit_splitters(samples: torch.Tensor, P: int, cfg: pgs_config, splitters_out: torch.Tensor,
                      model_out: torch.Tensor | None = None, stream=None) -> None:
    _check(load().pgs_fit_splitters(_ptr(samples), samples.numel(), P, _stream(stream), ctypes.byref(cfg),
                                    _ptr(splitters_out), _ptr(model_out)), "pgs_fit_splitters")


def pgs_get_stats(stats_dev: torch.Tensor, stream=None) -> dict:
    out = pgs_stats()
    _check(load().pgs_get_stats(_ptr(stats_dev), ctypes.byref(out), _stream(stream)), "pgs_get_stats")
    return out.as_dict()


STATS_BYTES = ctypes.sizeof(pgs_stats)


# ---------------------------------------------------------------------------
# Convenience layer on top of the C ABI (still marshalling only).
# ---------------------------------------------------------------------------

def as_device_keys(keys, dtype: str, device="cuda") -> torch.Tensor:
    """numpy uint32/uint64 (float32 as uint32 bits) -> device tensor of the same bits."""
    import numpy as np
    arr = np.ascontiguousarray(keys)
    view = arr.view(np.int64 if dtype == "u64" else np.int32)
    return torch.from_numpy(view).to(device)


def to_numpy_keys(t: torch.Tensor, dtype: str):
    import numpy as np
    a = t.cpu().numpy()
    return a.view(np.uint64 if dtype == "u64" else np.uint32)


def sort(keys: torch.Tensor, vals: torch.Tensor | None, P: int, dtype: str = "u32", out=None, device=None,
         **opts):
    """Sort a key/payload pair out of place; returns (keys, vals, info), info
    holding the bucket bounds and stats tensors (on the device).

    Device tensors go through pgs_sort_copy.  Host tensors go through
    pgs_sort_host (copies inside the library); `out` = (keys_out, vals_out)
    host tensors to fill, else fresh pinned ones are allocated.  The call
    returns once host outputs are complete."""
    host = not keys.is_cuda
    dev = torch.device(device or "cuda") if host else keys.device
    n = keys.numel()
    cfg = make_config(dtype=dtype, **opts)
    Peff = max(1, min(P, n)) if n else 1
    bounds = torch.empty(Peff + 1, dtype=torch.int64, device=dev)
    st = torch.zeros(STATS_BYTES, dtype=torch.uint8, device=dev)
    info = {"bucket_bounds": bounds, "stats": st}
    if host:
        nbytes = pgs_host_workspace_bytes(n, P, cfg)
        if nbytes == 0:
            raise PgsError(PGS_ERR_INVALID, "pgs_host_workspace_bytes")
        ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        cfg = make_config(dtype=dtype, workspace=ws, bucket_bounds=bounds, stats=st, **opts)
        if out is not None:
            ko, vo = out
        else:
            ko = torch.empty(keys.shape, dtype=keys.dtype, pin_memory=True)
            vo = torch.empty(vals.shape, dtype=vals.dtype, pin_memory=True) if vals is not None else None
        with torch.cuda.device(dev):
            pgs_sort_host(keys, vals, ko, vo, P, cfg)
            torch.cuda.current_stream().synchronize()
        return ko, vo, info
    ws = workspace(n, P, cfg, device=dev)
    cfg = make_config(dtype=dtype, workspace=ws, bucket_bounds=bounds, stats=st, **opts)
    kout = torch.empty_like(keys)
    vout = torch.empty_like(vals) if vals is not None else None
    pgs_sort_copy(keys, vals, kout, vout, P, cfg)
    return kout, vout, info
