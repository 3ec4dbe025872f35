"""Thin Python binding of libpandelos_gpu.so (the C ABI of include/pd.h).

Every function keeps the C name and only marshals arguments: numpy arrays or
torch tensors become pointers, handles stay opaque, and a non-OK status raises
``PdError`` with the library's message.  All computation happens in the CUDA
library; there is no Python or CPU fallback -- if the library cannot be built
or loaded, ``load()`` raises.

Device memory is taken from PyTorch's caching allocator (through the
library's allocator hooks) and work runs on PyTorch's current CUDA stream
unless another stream is given.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

PD_OK = 0
STATUS_NAMES = {0: "PD_OK", 1: "PD_ERR_ARG", 2: "PD_ERR_ALPHABET", 3: "PD_ERR_GENE_TOO_LONG",
                4: "PD_ERR_K_RANGE", 5: "PD_ERR_OOM", 6: "PD_ERR_BUDGET", 7: "PD_ERR_CUDA",
                8: "PD_ERR_TIMEOUT", 9: "PD_ERR_BUSY", 10: "PD_ERR_INTERNAL"}
PD_MAX_K = 8
PD_MAX_WINDOWS = 65535
PD_MAX_GENOMES = 4096
PD_NOALLOC_SCRATCH_BYTES = 32 << 20
PD_NOALLOC_MAX_ROWS = 32768
PD_NOALLOC_MAX_TARGETS = 32768
PD_NOALLOC_MAX_HITS = 1 << 20


class PdError(RuntimeError):
    def __init__(self, status: int, func: str, msg: str):
        super().__init__(f"{func}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ProfilesInfo(C.Structure):
    _fields_ = [("k", C.c_int), ("n_genes", C.c_uint32), ("n_genomes", C.c_uint32),
                ("n_windows", C.c_uint64), ("n_distinct", C.c_uint64), ("n_entries", C.c_uint64),
                ("max_posting", C.c_uint32), ("count_bits", C.c_uint32), ("device_bytes", C.c_uint64),
                ("alphabet", C.c_int), ("n_join", C.c_uint64)]


class HitsInfo(C.Structure):
    _fields_ = [("n_rows", C.c_uint32), ("n_hits", C.c_uint64), ("row_base", C.c_uint32),
                ("col_base", C.c_uint32), ("n_deferred", C.c_uint32), ("postings_walked", C.c_uint64)]


class Filter(C.Structure):
    _fields_ = [("theta_num", C.c_uint32), ("theta_den", C.c_uint32), ("tau_num", C.c_uint32),
                ("tau_den", C.c_uint32)]


class BatchTuning(C.Structure):
    _fields_ = [("max_chunk_windows", C.c_uint64), ("max_chunk_jobs", C.c_uint32), ("query_order", C.c_uint32),
                ("walk", C.c_uint32)]


class BatchInfo(C.Structure):
    _fields_ = [("n_jobs", C.c_uint32), ("n_chunks", C.c_uint32), ("n_rows", C.c_uint64), ("n_hits", C.c_uint64),
                ("n_bbh", C.c_uint64), ("postings_walked", C.c_uint64)]


class ReplyInfo(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("status", C.c_int32), ("snapshot_genomes", C.c_uint32),
                ("n_genes", C.c_uint32), ("tick_requests", C.c_uint32), ("n_hits", C.c_uint64),
                ("n_bbh", C.c_uint64), ("t_submit_ns", C.c_int64), ("t_start_ns", C.c_int64),
                ("t_done_ns", C.c_int64)]


class IndexInfo(C.Structure):
    _fields_ = [("k", C.c_int), ("n_genomes", C.c_uint32), ("n_genes", C.c_uint64), ("queued", C.c_uint32),
                ("max_tick_requests", C.c_uint32), ("device_bytes", C.c_uint64), ("budget", C.c_uint64),
                ("ticks", C.c_uint64), ("requests_done", C.c_uint64)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every exported function
_P = C.c_void_p
_PP = C.POINTER(C.c_void_p)
_SIGNATURES = [
    ("pd_ctx_create", C.c_int, [C.c_int, _P, ALLOC_FN, FREE_FN, _P, _PP]),
    ("pd_ctx_destroy", None, [_P]),
    ("pd_ctx_set_stream", C.c_int, [_P, _P]),
    ("pd_last_error", C.c_char_p, [_P]),
    ("pd_ctx_launch_count", C.c_uint64, [_P]),
    ("pd_ctx_set_timing", C.c_int, [_P, C.c_int]),
    ("pd_ctx_set_timing_filter", C.c_int, [_P, C.c_char_p]),
    ("pd_ctx_kernel_time", C.c_int, [_P, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_uint64)]),
    ("pd_ctx_reset_timing", C.c_int, [_P]),
    ("pd_choose_k", C.c_int, [C.c_uint64, C.c_int]),
    ("pd_build_profiles", C.c_int, [_P, _P, C.c_uint64, _P, C.c_uint32, _P, C.c_uint32, C.c_int, _PP]),
    ("pd_build_profiles_alphabet", C.c_int, [_P, _P, C.c_uint64, _P, C.c_uint32, _P, C.c_uint32, C.c_int, C.c_int,
                                             _PP]),
    ("pd_build_profiles_segmented", C.c_int, [_P, _P, C.c_uint64, _P, C.c_uint32, _P, C.c_uint32, _P, C.c_int,
                                              _PP]),
    ("pd_profiles_get_info", C.c_int, [_P, C.POINTER(ProfilesInfo)]),
    ("pd_profiles_copy_mv", C.c_int, [_P, _P, _P, _P, _P, _P]),
    ("pd_profiles_copy_index", C.c_int, [_P, _P, _P, _P, _P, _P]),
    ("pd_profiles_free", None, [_P]),
    ("pd_best_hits_all", C.c_int, [_P, _P, _PP]),
    ("pd_best_hits", C.c_int, [_P, _P, C.c_uint32, C.c_uint32, _PP]),
    ("pd_hits_get_info", C.c_int, [_P, C.POINTER(HitsInfo)]),
    ("pd_hits_copy", C.c_int, [_P, _P, _P, _P, _P, C.POINTER(C.c_uint64)]),
    ("pd_hits_free", None, [_P]),
    ("pd_bbh_all", C.c_int, [_P, _P, _P, _PP]),
    ("pd_bbh", C.c_int, [_P, _P, C.c_uint32, C.c_uint32, _PP]),
    ("pd_bbh_copy", C.c_int, [_P, _P, _P, _P, C.POINTER(C.c_uint64)]),
    ("pd_bbh_count", C.c_uint64, [_P]),
    ("pd_bbh_free", None, [_P]),
    ("pd_summin_pairs", C.c_int, [_P, _P, C.c_uint32, C.c_uint32, _P, _P, _P, C.POINTER(C.c_uint64)]),
    ("pd_bbh_batch", C.c_int, [_P, _P, C.c_uint64, _P, C.c_uint32, _P, C.c_uint32, _P, _P, C.c_uint32,
                               C.POINTER(BatchTuning), _PP]),
    ("pd_bbh_pairs", C.c_int, [_P, _P, _P, C.c_uint32, _PP]),
    ("pd_batch_get_info", C.c_int, [_P, C.POINTER(BatchInfo)]),
    ("pd_batch_autotune", C.c_int, [_P, _P, C.c_uint64, _P, C.c_uint32, _P, C.c_uint32, _P, _P, C.c_uint32,
                                    C.c_uint32, C.POINTER(BatchTuning), C.POINTER(C.c_double)]),
    ("pd_batch_copy_hits", C.c_int, [_P, _P, _P, _P, _P]),
    ("pd_batch_copy_bbh", C.c_int, [_P, _P, _P, _P, _P]),
    ("pd_batch_free", None, [_P]),
    ("pd_best_hits_all_filtered", C.c_int, [_P, _P, C.POINTER(Filter), _PP]),
    ("pd_best_hits_filtered", C.c_int, [_P, _P, C.c_uint32, C.c_uint32, C.POINTER(Filter), _PP]),
    ("pd_paralog_hits", C.c_int, [_P, _P, _PP]),
    ("pd_paralog_bbh", C.c_int, [_P, _P, _P, _PP]),
    ("pd_components", C.c_int, [_P, _P, _P, C.c_uint64, C.c_uint32, _P, C.POINTER(C.c_uint32)]),
    ("pd_families", C.c_int, [_P, _P, C.c_uint32, _P, C.POINTER(C.c_uint32)]),
    ("pd_index_create", C.c_int, [_P, _P, C.c_uint64, _P, C.c_uint32, _P, C.c_uint32, C.c_int, C.c_uint64, _PP]),
    ("pd_index_submit", C.c_int, [_P, _P, C.c_uint64, _P, C.c_uint32, C.POINTER(C.c_uint64)]),
    ("pd_index_poll", C.c_int, [_P, C.c_uint64, C.c_int, _PP]),
    ("pd_index_get_info", C.c_int, [_P, C.POINTER(IndexInfo)]),
    ("pd_index_hold", C.c_int, [_P, C.c_int]),
    ("pd_profiles_genome_ptr", C.c_int, [_P, _P]),
    ("pd_best_hits_shard", C.c_int, [_P, _P, C.c_uint32, C.c_uint32, _PP]),
    ("pd_summin_list", C.c_int, [_P, _P, _P, _P, C.c_uint64, _P, _P]),
    ("pd_ctx_set_symmetric", C.c_int, [_P, C.c_int]),
    ("pd_ctx_set_walk", C.c_int, [_P, C.c_uint32]),
    ("pd_hits_import", C.c_int, [_P, _P, C.c_uint32, _P, _P, _P, _P, _PP]),
    ("pd_index_genome_ptr", C.c_int, [_P, C.c_uint32, _P]),
    ("pd_index_free", None, [_P]),
    ("pd_reply_get_info", C.c_int, [_P, C.POINTER(ReplyInfo)]),
    ("pd_reply_error", C.c_char_p, [_P]),
    ("pd_reply_copy", C.c_int, [_P, _P, _P, _P, _P, _P]),
    ("pd_reply_free", None, [_P]),
    ("pd_best_hits_noalloc", C.c_int, [_P, _P, C.c_uint32, C.c_uint32, _P, _P, _P, C.c_uint64,
                                       C.POINTER(C.c_uint64)]),
]
EXPORTED = [s[0] for s in _SIGNATURES]


def library_path() -> str:
    return _build.LIB


def load(build: bool = True) -> C.CDLL:
    """Load libpandelos_gpu.so (building it first if needed); raises if impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libpandelos_gpu.so not found at {path}; build it with __graft_entry__.build()")
        lib = C.CDLL(path)
        for name, res, args in _SIGNATURES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(x):
    """Raw address of a numpy array or torch tensor (contiguous), or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to the library must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors passed to the library must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"cannot pass {type(x)} to the library")


def _check(ctx, st, func):
    if st != PD_OK:
        msg = _lib.pd_last_error(ctx.handle if ctx is not None else None)
        raise PdError(st, func, msg.decode() if msg else "")


# ---------------------------------------------------------------- context
class Ctx:
    """Owns a pd_ctx*; device memory comes from torch's caching allocator.

    on_alloc(nbytes) -> bool and on_free(ptr), if given, see every device
    allocation and release the library makes through this context (torch's
    allocator serves them).  on_alloc returning False refuses that
    allocation: the library then reports PD_ERR_OOM for the call.  Use them to
    account for or cap the library's device memory."""

    def __init__(self, device: int = 0, stream=None, use_torch_allocator: bool = True, on_alloc=None,
                 on_free=None):
        import torch
        lib = load()
        self.device = int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self._keep = []
        if use_torch_allocator:
            dev = self.device

            def _alloc(nbytes, strm, user):
                try:
                    if on_alloc is not None and on_alloc(int(nbytes)) is False:
                        return None
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, strm or 0)
                except Exception:
                    return None

            def _free(p, nbytes, strm, user):
                if on_free is not None:
                    on_free(p)
                torch.cuda.caching_allocator_delete(p)

            a, f = ALLOC_FN(_alloc), FREE_FN(_free)
            self._keep = [a, f]
        else:
            if on_alloc is not None or on_free is not None:
                raise ValueError("allocation observers need use_torch_allocator=True")
            a, f = ALLOC_FN(), FREE_FN()
        h = C.c_void_p()
        st = lib.pd_ctx_create(self.device, stream, a, f, None, C.byref(h))
        if st != PD_OK:
            raise PdError(st, "pd_ctx_create", "context creation failed")
        self.handle = h

    # Every handle made with this context must be freed before pd_ctx_destroy.
    # The garbage collector finalizes a reference cycle (a frame kept alive by
    # a caught exception's traceback) in no fixed order, so the context counts
    # its live handles and a close() that comes first waits for the last one.
    def _retain(self):
        self._live = getattr(self, "_live", 0) + 1

    def _release(self):
        self._live -= 1
        if self._live == 0 and getattr(self, "_closing", False):
            self._destroy()

    def _destroy(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.pd_ctx_destroy(self.handle)
            self.handle = None

    def close(self):
        self._closing = True
        if getattr(self, "_live", 0) == 0:
            self._destroy()

    def __del__(self):
        self.close()


def pd_ctx_create(device: int = 0, stream=None, use_torch_allocator: bool = True, on_alloc=None,
                  on_free=None) -> Ctx:
    return Ctx(device, stream, use_torch_allocator, on_alloc, on_free)


def pd_ctx_destroy(ctx: Ctx) -> None:
    ctx.close()


def pd_ctx_set_stream(ctx: Ctx, stream) -> None:
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(ctx, _lib.pd_ctx_set_stream(ctx.handle, s), "pd_ctx_set_stream")


def pd_last_error(ctx: Ctx) -> str:
    return _lib.pd_last_error(ctx.handle).decode()


def pd_ctx_launch_count(ctx: Ctx) -> int:
    return int(_lib.pd_ctx_launch_count(ctx.handle))


def pd_ctx_set_timing(ctx: Ctx, enable: bool) -> None:
    _check(ctx, _lib.pd_ctx_set_timing(ctx.handle, int(bool(enable))), "pd_ctx_set_timing")


def pd_ctx_set_symmetric(ctx: Ctx, enable: bool) -> None:
    """pd_best_hits_all walks each genome pair from one side (True, the
    default) or every genome from every query (False); same results."""
    _check(ctx, _lib.pd_ctx_set_symmetric(ctx.handle, 1 if enable else 0), "pd_ctx_set_symmetric")


PD_WALK_AUTO, PD_WALK_MERGE, PD_WALK_WARP = 0, 1, 2


def pd_ctx_set_walk(ctx: Ctx, mode: int) -> None:
    """Posting walk of the sum-min kernel for later Best Hit calls:
    PD_WALK_AUTO (from the build's join), PD_WALK_MERGE or PD_WALK_WARP; same
    results."""
    _check(ctx, _lib.pd_ctx_set_walk(ctx.handle, int(mode)), "pd_ctx_set_walk")


def pd_ctx_set_timing_filter(ctx: Ctx, name: str | None) -> None:
    """Time only launches of kernel `name` (None: every kernel)."""
    _check(ctx, _lib.pd_ctx_set_timing_filter(ctx.handle, name.encode() if name else None),
           "pd_ctx_set_timing_filter")


def pd_ctx_kernel_time(ctx: Ctx, name: str | None = None):
    """(milliseconds, launches) summed over kernel `name` (None: all)."""
    ms, n = C.c_double(0), C.c_uint64(0)
    _check(ctx, _lib.pd_ctx_kernel_time(ctx.handle, name.encode() if name else None, C.byref(ms), C.byref(n)),
           "pd_ctx_kernel_time")
    return ms.value, n.value


def pd_ctx_reset_timing(ctx: Ctx) -> None:
    _check(ctx, _lib.pd_ctx_reset_timing(ctx.handle), "pd_ctx_reset_timing")


def pd_choose_k(total_residues: int, alphabet: int = 20) -> int:
    return int(load().pd_choose_k(int(total_residues), int(alphabet)))


# ---------------------------------------------------------------- handles
class _Handle:
    _free_name = ""

    def __init__(self, ctx: Ctx, h: C.c_void_p):
        self.ctx = ctx
        self.handle = h
        ctx._retain()

    def free(self):
        if getattr(self, "handle", None) and _lib is not None:
            getattr(_lib, self._free_name)(self.handle)
            self.handle = None
            self.ctx._release()

    def __del__(self):
        self.free()


class Profiles(_Handle):
    _free_name = "pd_profiles_free"


class Hits(_Handle):
    _free_name = "pd_hits_free"


class BbhSet(_Handle):
    _free_name = "pd_bbh_free"


class Batch(_Handle):
    _free_name = "pd_batch_free"


class Index(_Handle):
    _free_name = "pd_index_free"


class Reply(_Handle):
    _free_name = "pd_reply_free"


def pd_build_profiles(ctx: Ctx, residues, gene_ptr, genome_ptr, k: int) -> Profiles:
    """residues uint8[N], gene_ptr int64[G+1], genome_ptr int32[n+1]: host or device."""
    n_res = int(residues.shape[0])
    n_genes = int(gene_ptr.shape[0]) - 1
    n_genomes = int(genome_ptr.shape[0]) - 1
    h = C.c_void_p()
    st = _lib.pd_build_profiles(ctx.handle, _ptr(residues), n_res, _ptr(gene_ptr), n_genes, _ptr(genome_ptr),
                                n_genomes, int(k), C.byref(h))
    _check(ctx, st, "pd_build_profiles")
    return Profiles(ctx, h)


PD_ALPHABET_AMINO = 20
PD_ALPHABET_NUCLEOTIDE = 4
PD_MAX_K_NUCLEOTIDE = 16


def pd_build_profiles_alphabet(ctx: Ctx, residues, gene_ptr, genome_ptr, alphabet: int, k: int) -> Profiles:
    """pd_build_profiles over 20 amino acids or 4 nucleotides (ACGT)."""
    n_res = int(residues.shape[0])
    h = C.c_void_p()
    st = _lib.pd_build_profiles_alphabet(ctx.handle, _ptr(residues), n_res, _ptr(gene_ptr), int(gene_ptr.shape[0]) - 1,
                                         _ptr(genome_ptr), int(genome_ptr.shape[0]) - 1, int(alphabet), int(k),
                                         C.byref(h))
    _check(ctx, st, "pd_build_profiles_alphabet")
    return Profiles(ctx, h)


def pd_build_profiles_segmented(ctx: Ctx, residues, gene_ptr, genome_ptr, genome_seg, k: int) -> Profiles:
    """pd_build_profiles with a segment per genome (genome_seg: host uint32[n]);
    genomes of different segments share no k-mer."""
    n_res = int(residues.shape[0])
    n_genes = int(gene_ptr.shape[0]) - 1
    n_genomes = int(genome_ptr.shape[0]) - 1
    seg = np.ascontiguousarray(genome_seg, dtype=np.uint32)
    h = C.c_void_p()
    st = _lib.pd_build_profiles_segmented(ctx.handle, _ptr(residues), n_res, _ptr(gene_ptr), n_genes,
                                          _ptr(genome_ptr), n_genomes, _ptr(seg), int(k), C.byref(h))
    _check(ctx, st, "pd_build_profiles_segmented")
    return Profiles(ctx, h)


def pd_profiles_get_info(prof: Profiles) -> ProfilesInfo:
    info = ProfilesInfo()
    _check(prof.ctx, _lib.pd_profiles_get_info(prof.handle, C.byref(info)), "pd_profiles_get_info")
    return info


def pd_profiles_genome_ptr(prof: Profiles):
    """Host int32 genome offsets (n_genomes+1) the profiles were built with."""
    out = np.zeros(pd_profiles_get_info(prof).n_genomes + 1, np.int32)
    _check(prof.ctx, _lib.pd_profiles_genome_ptr(prof.handle, _ptr(out)), "pd_profiles_genome_ptr")
    return out


def pd_profiles_copy_mv(ctx: Ctx, prof: Profiles):
    """(mv_ptr int64[G+1], codes uint64[E], counts uint32[E], La uint32[G]) on the host."""
    info = pd_profiles_get_info(prof)
    G, E = info.n_genes, info.n_entries
    mv_ptr = np.zeros(G + 1, np.int64)
    codes = np.zeros(max(E, 1), np.uint64)
    counts = np.zeros(max(E, 1), np.uint32)
    La = np.zeros(max(G, 1), np.uint32)
    _check(ctx, _lib.pd_profiles_copy_mv(ctx.handle, prof.handle, _ptr(mv_ptr), _ptr(codes), _ptr(counts),
                                         _ptr(La)), "pd_profiles_copy_mv")
    return mv_ptr, codes[:E], counts[:E], La[:G]


def pd_profiles_copy_index(ctx: Ctx, prof: Profiles):
    """(post_ptr int64[D+1], codes uint64[D], genes int32[E], counts uint32[E]) on the host."""
    info = pd_profiles_get_info(prof)
    D, E = info.n_distinct, info.n_entries
    post_ptr = np.zeros(D + 1, np.int64)
    codes = np.zeros(max(D, 1), np.uint64)
    genes = np.zeros(max(E, 1), np.int32)
    counts = np.zeros(max(E, 1), np.uint32)
    _check(ctx, _lib.pd_profiles_copy_index(ctx.handle, prof.handle, _ptr(post_ptr), _ptr(codes), _ptr(genes),
                                            _ptr(counts)), "pd_profiles_copy_index")
    return post_ptr, codes[:D], genes[:E], counts[:E]


def pd_best_hits_all(ctx: Ctx, prof: Profiles) -> Hits:
    h = C.c_void_p()
    _check(ctx, _lib.pd_best_hits_all(ctx.handle, prof.handle, C.byref(h)), "pd_best_hits_all")
    return Hits(ctx, h)


def pd_best_hits_shard(ctx: Ctx, prof: Profiles, shard: int, n_shards: int) -> Hits:
    """pd_best_hits_all restricted to shard `shard` of `n_shards` of the query
    genes (rows of other genes empty); the union over shards is the whole."""
    h = C.c_void_p()
    _check(ctx, _lib.pd_best_hits_shard(ctx.handle, prof.handle, int(shard), int(n_shards), C.byref(h)),
           "pd_best_hits_shard")
    return Hits(ctx, h)


def pd_hits_import(ctx: Ctx, prof: Profiles, pieces) -> Hits:
    """One Best Hit handle from CSR pieces [(row_ptr int64 [n_genes+1], cols
    int32 global ids ascending per row, s 32-bit), ...] (host or device), each
    gene's row non-empty in at most one piece."""
    G = pd_profiles_get_info(prof).n_genes
    pieces = list(pieces)
    n = len(pieces)
    if n == 0:
        raise ValueError("pd_hits_import: no pieces")
    rps, cls, ss, ns = (C.c_void_p * n)(), (C.c_void_p * n)(), (C.c_void_p * n)(), (C.c_uint64 * n)()
    for i, (rp, cols, s) in enumerate(pieces):
        if int(rp.shape[0]) != G + 1 or int(s.shape[0]) != int(cols.shape[0]):
            raise ValueError("pd_hits_import: row_ptr must have n_genes+1 entries and s one per column")
        k = int(cols.shape[0])
        rps[i], cls[i], ss[i], ns[i] = _ptr(rp), _ptr(cols) if k else None, _ptr(s) if k else None, k
    h = C.c_void_p()
    _check(ctx, _lib.pd_hits_import(ctx.handle, prof.handle, n, rps, cls, ss, ns, C.byref(h)), "pd_hits_import")
    return Hits(ctx, h)


def pd_best_hits(ctx: Ctx, prof: Profiles, gi: int, gj: int) -> Hits:
    h = C.c_void_p()
    _check(ctx, _lib.pd_best_hits(ctx.handle, prof.handle, int(gi), int(gj), C.byref(h)), "pd_best_hits")
    return Hits(ctx, h)


def pd_hits_get_info(hits: Hits) -> HitsInfo:
    info = HitsInfo()
    _check(hits.ctx, _lib.pd_hits_get_info(hits.handle, C.byref(info)), "pd_hits_get_info")
    return info


def pd_hits_copy(ctx: Ctx, hits: Hits, row_ptr=None, cols=None, s=None):
    """Copy Best Hits as CSR.  Without buffers, allocates host arrays and returns
    (row_ptr int64[n_rows+1], cols int32[n], s uint32[n])."""
    if row_ptr is None and cols is None and s is None:
        info = pd_hits_get_info(hits)
        row_ptr = np.zeros(info.n_rows + 1, np.int64)
        cols = np.zeros(max(info.n_hits, 1), np.int32)
        s = np.zeros(max(info.n_hits, 1), np.uint32)
        n = C.c_uint64(0)
        _check(ctx, _lib.pd_hits_copy(ctx.handle, hits.handle, _ptr(row_ptr), _ptr(cols), _ptr(s), C.byref(n)),
               "pd_hits_copy")
        return row_ptr, cols[:n.value], s[:n.value]
    n = C.c_uint64(0)
    _check(ctx, _lib.pd_hits_copy(ctx.handle, hits.handle, _ptr(row_ptr), _ptr(cols), _ptr(s), C.byref(n)),
           "pd_hits_copy")
    return int(n.value)


def pd_bbh_all(ctx: Ctx, prof: Profiles, hits: Hits) -> BbhSet:
    h = C.c_void_p()
    _check(ctx, _lib.pd_bbh_all(ctx.handle, prof.handle, hits.handle, C.byref(h)), "pd_bbh_all")
    return BbhSet(ctx, h)


def pd_bbh(ctx: Ctx, prof: Profiles, gi: int, gj: int) -> BbhSet:
    h = C.c_void_p()
    _check(ctx, _lib.pd_bbh(ctx.handle, prof.handle, int(gi), int(gj), C.byref(h)), "pd_bbh")
    return BbhSet(ctx, h)


def _filter(theta, tau):
    return Filter(int(theta[0]), int(theta[1]), int(tau[0]), int(tau[1]))


def pd_best_hits_all_filtered(ctx: Ctx, prof: Profiles, theta=(0, 1), tau=(0, 1)) -> Hits:
    """pd_best_hits_all with the theta (Eq. (6)) and tau (Eq. (7)) candidate
    filters, each a (numerator, denominator) fraction; numerator 0 = off."""
    h = C.c_void_p()
    f = _filter(theta, tau)
    _check(ctx, _lib.pd_best_hits_all_filtered(ctx.handle, prof.handle, C.byref(f), C.byref(h)),
           "pd_best_hits_all_filtered")
    return Hits(ctx, h)


def pd_best_hits_filtered(ctx: Ctx, prof: Profiles, gi: int, gj: int, theta=(0, 1), tau=(0, 1)) -> Hits:
    h = C.c_void_p()
    f = _filter(theta, tau)
    _check(ctx, _lib.pd_best_hits_filtered(ctx.handle, prof.handle, int(gi), int(gj), C.byref(f), C.byref(h)),
           "pd_best_hits_filtered")
    return Hits(ctx, h)


def pd_paralog_hits(ctx: Ctx, prof: Profiles) -> Hits:
    """Within-genome Best Hits of every gene (itself excluded)."""
    h = C.c_void_p()
    _check(ctx, _lib.pd_paralog_hits(ctx.handle, prof.handle, C.byref(h)), "pd_paralog_hits")
    return Hits(ctx, h)


def pd_paralog_bbh(ctx: Ctx, prof: Profiles, hits: Hits) -> BbhSet:
    """Mutual within-genome Best Hits (a < b, same genome)."""
    h = C.c_void_p()
    _check(ctx, _lib.pd_paralog_bbh(ctx.handle, prof.handle, hits.handle, C.byref(h)), "pd_paralog_bbh")
    return BbhSet(ctx, h)


def pd_bbh_count(bbh: BbhSet) -> int:
    return int(_lib.pd_bbh_count(bbh.handle))


def pd_bbh_copy(ctx: Ctx, bbh: BbhSet, a=None, b=None):
    """Copy pairs.  Without buffers returns a host int32 array [n, 2]."""
    if a is None and b is None:
        n = pd_bbh_count(bbh)
        a = np.zeros(max(n, 1), np.int32)
        b = np.zeros(max(n, 1), np.int32)
        _check(ctx, _lib.pd_bbh_copy(ctx.handle, bbh.handle, _ptr(a), _ptr(b), None), "pd_bbh_copy")
        return np.stack([a[:n], b[:n]], axis=1)
    n = C.c_uint64(0)
    _check(ctx, _lib.pd_bbh_copy(ctx.handle, bbh.handle, _ptr(a), _ptr(b), C.byref(n)), "pd_bbh_copy")
    return int(n.value)


def pd_summin_pairs(ctx: Ctx, prof: Profiles, gi: int, gj: int):
    """All (a, b, s) with s >= 1 between genomes gi and gj (local ids), host arrays."""
    n = C.c_uint64(0)
    _check(ctx, _lib.pd_summin_pairs(ctx.handle, prof.handle, int(gi), int(gj), None, None, None, C.byref(n)),
           "pd_summin_pairs")
    cnt = n.value
    a = np.zeros(max(cnt, 1), np.int32)
    b = np.zeros(max(cnt, 1), np.int32)
    s = np.zeros(max(cnt, 1), np.uint32)
    _check(ctx, _lib.pd_summin_pairs(ctx.handle, prof.handle, int(gi), int(gj), _ptr(a), _ptr(b), _ptr(s),
                                     C.byref(n)), "pd_summin_pairs")
    return a[:cnt], b[:cnt], s[:cnt]


def pd_summin_list(ctx: Ctx, prof: Profiles, a, b, s=None, den=None):
    """Sum-min and sum-max (Eq. (5)) of the gene pairs (a[i], b[i]) by merging
    their sorted multiplicity vectors.  a, b: uint32 global gene ids (host
    arrays or device tensors).  Without output buffers returns host arrays
    (s uint32, den uint32); with them (host or device, n entries) returns None."""
    n = int(a.shape[0])
    if int(b.shape[0]) != n:
        raise ValueError("pd_summin_list: a and b must have the same length")
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.uint32)
    if isinstance(b, np.ndarray):
        b = np.ascontiguousarray(b, dtype=np.uint32)
    ret = s is None and den is None
    if ret:
        s = np.zeros(max(n, 1), np.uint32)
        den = np.zeros(max(n, 1), np.uint32)
    _check(ctx, _lib.pd_summin_list(ctx.handle, prof.handle, _ptr(a) if n else None, _ptr(b) if n else None, n,
                                    _ptr(s), _ptr(den)), "pd_summin_list")
    if ret:
        return s[:n], den[:n]
    return None


def pd_best_hits_noalloc(ctx: Ctx, prof: Profiles, gi: int, gj: int, row_ptr, cols, s) -> int:
    """Best Hits of genome gi against gj into caller-owned device tensors, with
    no device allocation by the library (for callers that cannot allocate while
    they run).  row_ptr: int64 [|G_gi|+1]; cols: int32 [capacity]; s: uint32 or
    int32 [capacity], all CUDA tensors on ctx's device.  Returns the number of
    entries written."""
    import torch
    gptr = pd_profiles_genome_ptr(prof)
    n_rows = int(gptr[gi + 1] - gptr[gi]) if 0 <= gi < len(gptr) - 1 else 0
    for name, t in (("row_ptr", row_ptr), ("cols", cols), ("s", s)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device.index != ctx.device:
            raise ValueError(f"pd_best_hits_noalloc: {name} must be a CUDA tensor on device {ctx.device}")
    if row_ptr.dtype != torch.int64 or row_ptr.numel() < n_rows + 1:
        raise ValueError(f"pd_best_hits_noalloc: row_ptr must be int64 with at least {n_rows + 1} entries")
    if cols.dtype != torch.int32 or s.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)):
        raise ValueError("pd_best_hits_noalloc: cols must be int32 and s 32-bit")
    n = C.c_uint64(0)
    cap = min(int(cols.numel()), int(s.numel()))
    _check(ctx, _lib.pd_best_hits_noalloc(ctx.handle, prof.handle, int(gi), int(gj), _ptr(row_ptr), _ptr(cols),
                                          _ptr(s), cap, C.byref(n)), "pd_best_hits_noalloc")
    return int(n.value)


def pd_bbh_batch(ctx: Ctx, residues, gene_ptr, genome_ptr, jobs, job_k, max_chunk_windows: int = 0,
                 max_chunk_jobs: int = 0, query_order: int = 0, walk: int = 0) -> Batch:
    """Best Hits (both directions) and BBH of many genome-pair jobs: jobs is a
    host array [n_jobs, 2] of genome indices, job_k the k of each job."""
    n_res = int(residues.shape[0])
    n_genes = int(gene_ptr.shape[0]) - 1
    n_genomes = int(genome_ptr.shape[0]) - 1
    jb = np.ascontiguousarray(jobs, dtype=np.uint32).reshape(-1)
    kk = np.ascontiguousarray(job_k, dtype=np.int32)
    if jb.shape[0] != 2 * kk.shape[0]:
        raise ValueError("jobs must have two genome indices per entry of job_k")
    tun = BatchTuning(int(max_chunk_windows), int(max_chunk_jobs), int(query_order), int(walk))
    h = C.c_void_p()
    st = _lib.pd_bbh_batch(ctx.handle, _ptr(residues), n_res, _ptr(gene_ptr), n_genes, _ptr(genome_ptr), n_genomes,
                           _ptr(jb) if jb.size else None, _ptr(kk) if kk.size else None, int(kk.shape[0]),
                           C.byref(tun), C.byref(h))
    _check(ctx, st, "pd_bbh_batch")
    return Batch(ctx, h)


def pd_bbh_pairs(ctx: Ctx, prof: Profiles, jobs) -> Batch:
    """Best Hits both ways and BBH of many genome pairs [n_jobs, 2] of one
    profiled dataset, in one launch sequence (pd_batch result layout)."""
    jb = np.ascontiguousarray(jobs, dtype=np.uint32).reshape(-1)
    h = C.c_void_p()
    _check(ctx, _lib.pd_bbh_pairs(ctx.handle, prof.handle, _ptr(jb) if jb.size else None, jb.size // 2,
                                  C.byref(h)), "pd_bbh_pairs")
    return Batch(ctx, h)


def pd_batch_autotune(ctx: Ctx, residues, gene_ptr, genome_ptr, jobs, job_k, n_sample: int = 0):
    """Time candidate tunings on the first n_sample jobs; returns (dict of the
    fastest tuning, usable as pd_bbh_batch keywords, ms per sampled job)."""
    jb = np.ascontiguousarray(jobs, dtype=np.uint32).reshape(-1)
    kk = np.ascontiguousarray(job_k, dtype=np.int32)
    best = BatchTuning()
    ms = C.c_double(0)
    _check(ctx, _lib.pd_batch_autotune(ctx.handle, _ptr(residues), int(residues.shape[0]), _ptr(gene_ptr),
                                       int(gene_ptr.shape[0]) - 1, _ptr(genome_ptr), int(genome_ptr.shape[0]) - 1,
                                       _ptr(jb), _ptr(kk), int(kk.shape[0]), int(n_sample), C.byref(best),
                                       C.byref(ms)), "pd_batch_autotune")
    return ({"max_chunk_windows": int(best.max_chunk_windows), "max_chunk_jobs": int(best.max_chunk_jobs),
             "query_order": int(best.query_order), "walk": int(best.walk)}, float(ms.value))


def pd_batch_get_info(batch: Batch) -> BatchInfo:
    info = BatchInfo()
    _check(batch.ctx, _lib.pd_batch_get_info(batch.handle, C.byref(info)), "pd_batch_get_info")
    return info


def pd_batch_copy_hits(ctx: Ctx, batch: Batch, row_ptr=None, cols=None, s=None):
    """Best Hits of all jobs as one CSR (rows: genes of A then B per job;
    columns local to the partner genome).  Without buffers returns host arrays."""
    if row_ptr is None and cols is None and s is None:
        info = pd_batch_get_info(batch)
        row_ptr = np.zeros(info.n_rows + 1, np.int64)
        cols = np.zeros(max(info.n_hits, 1), np.int32)
        s = np.zeros(max(info.n_hits, 1), np.uint32)
        _check(ctx, _lib.pd_batch_copy_hits(ctx.handle, batch.handle, _ptr(row_ptr), _ptr(cols), _ptr(s)),
               "pd_batch_copy_hits")
        return row_ptr, cols[:info.n_hits], s[:info.n_hits]
    _check(ctx, _lib.pd_batch_copy_hits(ctx.handle, batch.handle, _ptr(row_ptr), _ptr(cols), _ptr(s)),
           "pd_batch_copy_hits")
    return None


def pd_batch_copy_bbh(ctx: Ctx, batch: Batch, job_ptr=None, a=None, b=None):
    """BBH pairs of all jobs: (job_ptr int64[n_jobs+1], pairs int32[n, 2]) with
    a local in A and b local in B.  Without buffers returns host arrays."""
    if job_ptr is None and a is None and b is None:
        info = pd_batch_get_info(batch)
        job_ptr = np.zeros(info.n_jobs + 1, np.int64)
        a = np.zeros(max(info.n_bbh, 1), np.int32)
        b = np.zeros(max(info.n_bbh, 1), np.int32)
        _check(ctx, _lib.pd_batch_copy_bbh(ctx.handle, batch.handle, _ptr(job_ptr), _ptr(a), _ptr(b)),
               "pd_batch_copy_bbh")
        return job_ptr, np.stack([a[:info.n_bbh], b[:info.n_bbh]], axis=1)
    _check(ctx, _lib.pd_batch_copy_bbh(ctx.handle, batch.handle, _ptr(job_ptr), _ptr(a), _ptr(b)),
           "pd_batch_copy_bbh")
    return None


# ---------------------------------------------------------------- served index
def _check_status(st, func, msg=""):
    if st != PD_OK:
        raise PdError(st, func, msg)


def pd_index_create(ctx: Ctx, residues, gene_ptr, genome_ptr, k: int, hbm_budget: int) -> Index:
    """Resident index over a dataset (host or device arrays) at a fixed k,
    with a worker that answers submitted genomes within hbm_budget bytes."""
    h = C.c_void_p()
    st = _lib.pd_index_create(ctx.handle, _ptr(residues), int(residues.shape[0]), _ptr(gene_ptr),
                              int(gene_ptr.shape[0]) - 1, _ptr(genome_ptr), int(genome_ptr.shape[0]) - 1, int(k),
                              int(hbm_budget), C.byref(h))
    _check(ctx, st, "pd_index_create")
    return Index(ctx, h)


def pd_index_submit(index: Index, residues, gene_ptr) -> int:
    """Queue one genome (host uint8 residues, int64 gene_ptr); returns its ticket."""
    res = np.ascontiguousarray(residues, dtype=np.uint8)
    gp = np.ascontiguousarray(gene_ptr, dtype=np.int64)
    t = C.c_uint64(0)
    _check_status(_lib.pd_index_submit(index.handle, _ptr(res) if res.size else None, int(res.shape[0]), _ptr(gp),
                                       int(gp.shape[0]) - 1, C.byref(t)), "pd_index_submit")
    return int(t.value)


def pd_index_poll(index: Index, ticket: int, wait_ms: int = -1) -> Reply:
    """The answer of a request (waits up to wait_ms; negative = no limit)."""
    h = C.c_void_p()
    _check_status(_lib.pd_index_poll(index.handle, int(ticket), int(wait_ms), C.byref(h)), "pd_index_poll")
    return Reply(index.ctx, h)


def pd_index_get_info(index: Index) -> IndexInfo:
    info = IndexInfo()
    _check_status(_lib.pd_index_get_info(index.handle, C.byref(info)), "pd_index_get_info")
    return info


def pd_index_hold(index: Index, hold: bool) -> None:
    """Pause (True) or resume (False) the admission of queued requests."""
    _check_status(_lib.pd_index_hold(index.handle, 1 if hold else 0), "pd_index_hold")


def pd_index_genome_ptr(index: Index, n_genomes: int):
    out = np.zeros(int(n_genomes) + 1, np.int32)
    _check_status(_lib.pd_index_genome_ptr(index.handle, int(n_genomes), _ptr(out)), "pd_index_genome_ptr")
    return out


def pd_reply_get_info(reply: Reply) -> ReplyInfo:
    info = ReplyInfo()
    _check_status(_lib.pd_reply_get_info(reply.handle, C.byref(info)), "pd_reply_get_info")
    return info


def pd_reply_copy(reply: Reply):
    """(row_ptr int64[n_genes+1], cols int32 resident gene ids, s uint32,
    bbh int32[n, 2] = (gene of the request, resident gene)); raises PdError if
    the request failed."""
    info = pd_reply_get_info(reply)
    if info.status != PD_OK:
        msg = _lib.pd_reply_error(reply.handle)
        raise PdError(info.status, "pd_reply_copy", msg.decode() if msg else "")
    rp = np.zeros(info.n_genes + 1, np.int64)
    cols = np.zeros(max(info.n_hits, 1), np.int32)
    s = np.zeros(max(info.n_hits, 1), np.uint32)
    a = np.zeros(max(info.n_bbh, 1), np.int32)
    b = np.zeros(max(info.n_bbh, 1), np.int32)
    _check_status(_lib.pd_reply_copy(reply.handle, _ptr(rp), _ptr(cols), _ptr(s), _ptr(a), _ptr(b)), "pd_reply_copy")
    return rp, cols[:info.n_hits], s[:info.n_hits], np.stack([a[:info.n_bbh], b[:info.n_bbh]], axis=1)


# ---------------------------------------------------------------- families
def pd_components(ctx: Ctx, a, b, n_nodes: int):
    """Connected components of the graph with edges (a[e], b[e]) (host or
    device int32): (labels int32[n_nodes] on the host, n_components)."""
    aa = a if hasattr(a, "data_ptr") else np.ascontiguousarray(a, dtype=np.int32)
    bb = b if hasattr(b, "data_ptr") else np.ascontiguousarray(b, dtype=np.int32)
    n_edges = int(aa.shape[0])
    lab = np.zeros(max(int(n_nodes), 1), np.int32)
    n = C.c_uint32(0)
    _check(ctx, _lib.pd_components(ctx.handle, _ptr(aa) if n_edges else None, _ptr(bb) if n_edges else None, n_edges,
                                   int(n_nodes), _ptr(lab), C.byref(n)), "pd_components")
    return lab[:int(n_nodes)], int(n.value)


def pd_families(ctx: Ctx, bbh: BbhSet, n_genes: int):
    """Gene families of an all-pairs BBH set: (labels int32[n_genes], count)."""
    lab = np.zeros(max(int(n_genes), 1), np.int32)
    n = C.c_uint32(0)
    _check(ctx, _lib.pd_families(ctx.handle, bbh.handle, int(n_genes), _ptr(lab), C.byref(n)), "pd_families")
    return lab[:int(n_genes)], int(n.value)
