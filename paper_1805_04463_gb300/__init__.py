"""GB300-native causal-set interval abundances and Benincasa-Dowker action.

Thin Python binding over the C ABI declared in include/cs.h (the compiled
library libcausetgb.so, CUDA for sm_103a).  Every function here only
marshals arguments: buffers are torch tensors (device memory and streams
come from PyTorch), and every step of the computation runs in the library's
kernels.  There is no CPU fallback: if the library is missing or cannot load,
every call raises CsError.

Reference: W. J. Cunningham, "High Performance Algorithms for Quantum Gravity
and Cosmology" (arXiv:1805.04463), Chapter "Causal Set Action".
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = [
    "KIND_2D_ORDER", "KIND_2D_DIAMOND", "KIND_4D_DIAMOND", "KIND_3D_DIAMOND", "KIND_2D_DS_SLAB", "KIND_2D_SQUARE", "KIND_2D_CYLINDER", "PATH_AUTO", "PATH_POPC", "PATH_MMA", "PATH_MMA4",
    "CsError", "lib", "dim", "coords_bytes", "row_words", "bitset_bytes", "hist_len",
    "sprinkle_workspace_bytes", "interval_abundance_workspace", "resolved_path", "action_workspace_bytes",
    "set_auto_paths", "get_auto_paths", "set_auto_memory_limit", "get_auto_memory_limit",
    "set_auto_tiles", "get_auto_tiles", "set_batch_tuning", "get_batch_tuning",
    "sprinkle", "sprinkle_noalloc", "causal_matrix", "layer_sums", "dalembertian", "interval_abundance", "workspace_status", "action", "action_device",
    "evaluate", "Buffers", "allocate", "run", "SetDesc", "Batch", "CountJob", "count_items",
    "operands_bytes", "prepare_operands", "peak_probe", "count_jobs", "degrees", "sparse_relations", "longest_chain", "greedy_antichain", "BATCH_MAX_N", "FAULT_ALLOC", "FAULT_LAUNCH", "selftest_wait",
    "inject_fault",
]

KIND_2D_ORDER, KIND_2D_DIAMOND, KIND_4D_DIAMOND, KIND_3D_DIAMOND, KIND_2D_DS_SLAB = 0, 1, 2, 3, 4
KIND_2D_SQUARE, KIND_2D_CYLINDER = 5, 6
PATH_AUTO, PATH_POPC, PATH_MMA, PATH_MMA4 = 0, 1, 2, 3
PENDING = 1  # CS_PENDING: polled work still running
FAULT_ALLOC, FAULT_LAUNCH = 1, 2
BATCH_MAX_N = 8192  # CS_BATCH_MAX_N: largest set a batch takes
KIND_NAMES = {KIND_2D_ORDER: "2d_order", KIND_2D_DIAMOND: "2d_diamond", KIND_4D_DIAMOND: "4d_diamond",
              KIND_3D_DIAMOND: "3d_diamond", KIND_2D_DS_SLAB: "2d_ds_slab", KIND_2D_SQUARE: "2d_square",
              KIND_2D_CYLINDER: "2d_cylinder"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "libcausetgb.so")
_lock = threading.Lock()
_lib = None


class CsError(RuntimeError):
    """A non-zero cs_status from the library, or the library is unavailable."""

    def __init__(self, status, what=""):
        self.status = status
        msg = status if isinstance(status, str) else f"{what}: status {status}"
        if not isinstance(status, str) and _lib is not None:
            msg += " (" + _lib.cs_strerror(status).decode() + ")"
            if status == -3:  # CS_ECUDA: name the CUDA error behind it
                msg += ": " + _lib.cs_last_cuda_error().decode()
        super().__init__(msg)


def lib() -> ctypes.CDLL:
    """Load libcausetgb.so (built by paper_1805_04463_gb300.build); raise if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIBPATH):
            raise CsError(f"{LIBPATH} is missing: build it with paper_1805_04463_gb300.build.build() "
                          "(there is no CPU fallback)")
        L = ctypes.CDLL(LIBPATH)
        i32, i64, u64, sz, vp, dp = (ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t,
                                     ctypes.c_void_p, ctypes.POINTER(ctypes.c_double))
        sig = {
            "cs_dim": ([i32], i32),
            "cs_coords_bytes": ([i32, i64], sz),
            "cs_row_words": ([i64], i64),
            "cs_bitset_bytes": ([i64], sz),
            "cs_hist_len": ([i64], i64),
            "cs_sprinkle_workspace_bytes": ([i32, i64], sz),
            "cs_sprinkle": ([i32, i64, u64, vp, vp, sz, vp], i32),
            "cs_causal_matrix": ([i32, i64, vp, vp, i64, vp], i32),
            "cs_interval_abundance_workspace": ([i64, i32], sz),
            "cs_mma4_band_panels": ([i64, sz], i64),
            "cs_mma4_band_cover": ([i64, i64, i32, vp], i64),
            "cs_resolved_path": ([i64, i32], i32),
            "cs_set_auto_paths": ([vp, vp, i32], i32),
            "cs_get_auto_paths": ([vp, vp, i32], i32),
            "cs_set_auto_memory_limit": ([sz], i32),
            "cs_set_auto_tiles": ([vp, vp, i32], i32),
            "cs_get_auto_tiles": ([vp, vp, i32], i32),
            "cs_set_batch_tuning": ([i32, i32], i32),
            "cs_get_batch_tuning": ([ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], i32),
            "cs_get_auto_memory_limit": ([], sz),
            "cs_interval_abundance": ([i64, vp, i64, vp, i32, vp, sz, vp], i32),
            "cs_workspace_status": ([vp, vp], i32),
            "cs_layer_sums": ([i64, vp, i64, vp, i32, vp, i32, vp, vp, sz, vp], i32),
            "cs_dalembertian": ([i32, i64, vp, vp, i32, ctypes.c_double, vp, vp], i32),
            "cs_action": ([i32, i64, vp, i64, ctypes.c_double, dp, ctypes.POINTER(ctypes.c_int64)], i32),
            "cs_action_workspace_bytes": ([], sz),
            "cs_action_device": ([i32, i64, vp, i64, vp, i32, vp, vp, vp, sz, vp], i32),
            "cs_evaluate": ([i32, i64, u64, vp, i32, vp, i32, vp, vp, vp, vp], i32),
            "cs_sprinkle_noalloc": ([i32, i64, u64, vp, vp], i32),
            "cs_batch_workspace_bytes": ([vp, i32, i32], sz),
            "cs_batch_hist_len": ([vp, i32], i64),
            "cs_batch_create": ([vp, i32, i32, vp, sz, ctypes.POINTER(ctypes.c_void_p), vp], i32),
            "cs_batch_launch": ([vp, vp, i32, vp, vp, vp, vp], i32),
            "cs_batch_path": ([vp], i32),
            "cs_batch_poll": ([vp], i32),
            "cs_batch_destroy": ([vp], None),
            "cs_count_items": ([i64, i32], i64),
            "cs_operands_bytes": ([i64, i32], sz),
            "cs_prepare_operands": ([i64, i32, vp, i64, vp, sz, vp], i32),
            "cs_count_jobs_table_bytes": ([i32, i32], sz),
            "cs_count_jobs_workspace_bytes": ([i32, i32], sz),
            "cs_count_jobs": ([vp, i32, i32, vp, vp, sz, vp], i32),
            "cs_degrees": ([i64, vp, i64, vp, vp, vp], i32),
            "cs_sparse_workspace_bytes": ([i64], ctypes.c_size_t),
            "cs_sparse_offsets": ([i64, vp, i64, i32, vp, vp, ctypes.c_size_t, vp], i32),
            "cs_sparse_columns": ([i64, vp, i64, i32, vp, vp, i64, vp, ctypes.c_size_t, vp], i32),
            "cs_chain_workspace_bytes": ([i64], ctypes.c_size_t),
            "cs_longest_chain": ([i64, vp, i64, i64, i64, ctypes.POINTER(ctypes.c_int64), vp, ctypes.c_size_t, vp],
                                 i32),
            "cs_greedy_antichain": ([i64, vp, i64, i64, vp, ctypes.POINTER(ctypes.c_int64), vp, ctypes.c_size_t,
                                     vp], i32),
            "cs_selftest_wait": ([vp, ctypes.c_double, i32, vp], i32),
            "cs_inject_fault": ([i32, i32], i32),
            "cs_strerror": ([i32], ctypes.c_char_p),
            "cs_version": ([], ctypes.c_char_p),
            "cs_last_cuda_error": ([], ctypes.c_char_p),
            "cs_peak_probe": ([i32, i64, vp, dp], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return L


def _check(rc, what):
    if rc != 0:
        raise CsError(rc, what)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def _ptr(t):
    return None if t is None else t.data_ptr()


def _nbytes(t):
    return t.numel() * t.element_size()


# ----------------------------------------------------------------- layouts

def dim(kind: int) -> int:
    return lib().cs_dim(kind)


def coords_bytes(kind: int, n: int) -> int:
    return lib().cs_coords_bytes(kind, n)


def row_words(n: int) -> int:
    return lib().cs_row_words(n)


def bitset_bytes(n: int) -> int:
    return lib().cs_bitset_bytes(n)


def hist_len(n: int) -> int:
    return lib().cs_hist_len(n)


def sprinkle_workspace_bytes(kind: int, n: int) -> int:
    return lib().cs_sprinkle_workspace_bytes(kind, n)


def interval_abundance_workspace(n: int, path: int = PATH_AUTO) -> int:
    return lib().cs_interval_abundance_workspace(n, path)


def mma4_band_panels(n: int, workspace_bytes: int) -> int:
    """Supertile rows per band of the FP4 count with this workspace: (n + 255) // 256
    when the whole operand matrix fits, 0 when not even one-panel bands do."""
    return lib().cs_mma4_band_panels(n, workspace_bytes)


def mma4_band_cover(n: int, panels: int, raster: int = 8):
    """(items, counts): the FP4 count's work items over all bands of `panels`
    supertile rows, and how many decode to each supertile (si, sj) (host only)."""
    import numpy as np
    nsb = (n + 255) // 256
    counts = np.zeros((nsb, nsb), dtype=np.int64)
    items = lib().cs_mma4_band_cover(n, panels, raster, counts.ctypes.data_as(ctypes.c_void_p))
    return items, counts


def resolved_path(n: int, path: int = PATH_AUTO) -> int:
    """PATH_POPC, PATH_MMA or PATH_MMA4: the kernel cs_interval_abundance runs for (n, path)."""
    return lib().cs_resolved_path(n, path)


def set_auto_paths(table):
    """Install the CS_PATH_AUTO table: sequence of (n_min, path), n_min from 0 upward."""
    n = (ctypes.c_int64 * len(table))(*[int(a) for a, _ in table])
    p = (ctypes.c_int * len(table))(*[int(b) for _, b in table])
    _check(lib().cs_set_auto_paths(n, p, len(table)), "cs_set_auto_paths")


def get_auto_paths():
    cnt = lib().cs_get_auto_paths(None, None, 0)
    n = (ctypes.c_int64 * cnt)()
    p = (ctypes.c_int * cnt)()
    lib().cs_get_auto_paths(n, p, cnt)
    return [(int(n[i]), int(p[i])) for i in range(cnt)]


def set_auto_tiles(table):
    """cs_set_auto_tiles: raster side per size bucket of the single-set tensor counts,
    a sequence of (n_min, raster), n_min from 0 upward."""
    n = (ctypes.c_int64 * len(table))(*[int(a) for a, _ in table])
    r = (ctypes.c_int * len(table))(*[int(b) for _, b in table])
    _check(lib().cs_set_auto_tiles(n, r, len(table)), "cs_set_auto_tiles")


def get_auto_tiles():
    cnt = lib().cs_get_auto_tiles(None, None, 0)
    n = (ctypes.c_int64 * cnt)()
    r = (ctypes.c_int * cnt)()
    lib().cs_get_auto_tiles(n, r, cnt)
    return [(int(n[i]), int(r[i])) for i in range(cnt)]


def set_batch_tuning(path=PATH_AUTO, max_run=16):
    """cs_set_batch_tuning: the path AUTO means for batches and count jobs, and the
    multi-set queue's run length."""
    _check(lib().cs_set_batch_tuning(int(path), int(max_run)), "cs_set_batch_tuning")


def get_batch_tuning():
    p, r = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().cs_get_batch_tuning(ctypes.byref(p), ctypes.byref(r)), "cs_get_batch_tuning")
    return p.value, r.value


def set_auto_memory_limit(nbytes: int = 0):
    """cs_set_auto_memory_limit: device bytes CS_PATH_AUTO may plan into (0 = 90% of the device)."""
    _check(lib().cs_set_auto_memory_limit(int(nbytes)), "cs_set_auto_memory_limit")


def get_auto_memory_limit() -> int:
    return lib().cs_get_auto_memory_limit()


def action_workspace_bytes() -> int:
    return lib().cs_action_workspace_bytes()


# ------------------------------------------------------------- entry points

def sprinkle(kind, n, seed, coords, workspace, stream=None):
    """cs_sprinkle: time-sorted int32 coordinates (dim, n) into `coords`."""
    _check(lib().cs_sprinkle(kind, n, seed, _ptr(coords), _ptr(workspace), _nbytes(workspace), _stream(stream)),
           "cs_sprinkle")


def sprinkle_noalloc(kind, n, seed, coords, stream=None):
    """cs_sprinkle_noalloc: as sprinkle(), with no workspace and no allocation (n <= 262144)."""
    _check(lib().cs_sprinkle_noalloc(kind, n, seed, _ptr(coords), _stream(stream)), "cs_sprinkle_noalloc")


def causal_matrix(kind, n, coords, bits, stream=None):
    """cs_causal_matrix: symmetric row bitsets (n, row_words) into `bits` (int64 storage)."""
    _check(lib().cs_causal_matrix(kind, n, _ptr(coords), _ptr(bits), bits.shape[-1], _stream(stream)),
           "cs_causal_matrix")


def interval_abundance(n, bits, hist, path=PATH_AUTO, workspace=None, stream=None):
    """cs_interval_abundance: N_k histogram (int64, hist_len(n)) into `hist`."""
    _check(lib().cs_interval_abundance(n, _ptr(bits), bits.shape[-1], _ptr(hist), path, _ptr(workspace),
                                       _nbytes(workspace), _stream(stream)), "cs_interval_abundance")


def layer_sums(n, bits, hist, layer, kmax, phi=None, path=PATH_AUTO, workspace=None, stream=None):
    """cs_layer_sums: histogram plus d'Alembertian layer sums layer[(kmax+1), n] (float64)."""
    _check(lib().cs_layer_sums(n, _ptr(bits), bits.shape[-1], _ptr(hist), path, _ptr(phi), kmax, _ptr(layer),
                               _ptr(workspace), _nbytes(workspace), _stream(stream)), "cs_layer_sums")


def dalembertian(dim_, n, layer, out, ell=1.0, phi=None, stream=None):
    """cs_dalembertian: B phi(j) for every element into the float64 tensor `out`."""
    _check(lib().cs_dalembertian(dim_, n, _ptr(phi), _ptr(layer), layer.shape[0] - 1, float(ell), _ptr(out),
                                 _stream(stream)), "cs_dalembertian")


def workspace_status(workspace, stream=None) -> int:
    """cs_workspace_status: in-kernel status of the last call on this workspace (synchronising)."""
    return lib().cs_workspace_status(_ptr(workspace), _stream(stream))


def action(dim_, n, hist, eps=0.0):
    """cs_action on a host int64 numpy histogram: (S, bracket)."""
    import numpy as np
    h = np.ascontiguousarray(hist, dtype=np.int64)
    out = ctypes.c_double(0.0)
    br = ctypes.c_int64(0)
    _check(lib().cs_action(dim_, n, h.ctypes.data if h.size else None, h.size, float(eps), ctypes.byref(out),
                           ctypes.byref(br)), "cs_action")
    return out.value, br.value


def action_device(dim_, n, hist, eps, out, bracket, workspace, stream=None):
    """cs_action_device: actions for each eps in `eps` into the float64 tensor `out`."""
    arr = (ctypes.c_double * len(eps))(*[float(e) for e in eps])
    _check(lib().cs_action_device(dim_, n, _ptr(hist), hist.numel(), ctypes.cast(arr, ctypes.c_void_p), len(eps),
                                  _ptr(out), _ptr(bracket), _ptr(workspace), _nbytes(workspace), _stream(stream)),
           "cs_action_device")


def evaluate(kind, n, seed=0, coords_host=None, path=PATH_AUTO, eps=(), stream=None, hist_out=None):
    """cs_evaluate from host buffers: returns (hist numpy int64, actions list, bracket).

    coords_host: optional numpy int32 (dim, n) array (pinned or pageable); when None the
    set is sprinkled on the device from (kind, n, seed).
    """
    import numpy as np
    hl = hist_len(n)
    hist = hist_out if hist_out is not None else np.zeros(hl, dtype=np.int64)
    acts = np.zeros(max(len(eps), 1), dtype=np.float64)
    br = ctypes.c_int64(0)
    arr = (ctypes.c_double * max(len(eps), 1))(*([float(e) for e in eps] or [0.0]))
    cptr = None
    if coords_host is not None:
        assert coords_host.dtype == np.int32 and coords_host.flags["C_CONTIGUOUS"]
        cptr = coords_host.ctypes.data
    _check(lib().cs_evaluate(kind, n, seed, cptr, path, ctypes.cast(arr, ctypes.c_void_p), len(eps),
                             hist.ctypes.data, acts.ctypes.data, ctypes.byref(br), _stream(stream)),
           "cs_evaluate")
    return hist, [float(x) for x in acts[:len(eps)]], br.value


# ---------------------------------------------------- device buffer helper

class Buffers:
    """Device buffers for one causal set of `kind` and size n (torch tensors)."""

    def __init__(self, kind, n, device="cuda", path=PATH_AUTO):
        import torch
        self.kind, self.n, self.path = kind, n, path
        self.dim = dim(kind)
        self.rw = row_words(n)
        self.coords = torch.empty((self.dim, n), dtype=torch.int32, device=device)
        self.bits = torch.empty((n, self.rw), dtype=torch.int64, device=device)
        self.hist = torch.empty(hist_len(n), dtype=torch.int64, device=device)
        ws = max(sprinkle_workspace_bytes(kind, n), interval_abundance_workspace(n, path), action_workspace_bytes())
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=device)
        self.actions = torch.empty(16, dtype=torch.float64, device=device)
        self.bracket = torch.empty(1, dtype=torch.int64, device=device)


def allocate(kind, n, device="cuda", path=PATH_AUTO) -> Buffers:
    return Buffers(kind, n, device, path)


def run(buf: Buffers, seed: int, eps=(0.0,), stream=None, sprinkle_=True):
    """One whole pass on device buffers: sprinkle, relate, count, actions (all async)."""
    if sprinkle_:
        sprinkle(buf.kind, buf.n, seed, buf.coords, buf.workspace, stream)
    causal_matrix(buf.kind, buf.n, buf.coords, buf.bits, stream)
    interval_abundance(buf.n, buf.bits, buf.hist, buf.path, buf.workspace, stream)
    if eps:
        action_device(buf.dim, buf.n, buf.hist, list(eps), buf.actions, buf.bracket, buf.workspace, stream)


# ------------------------------------------------------- batched ensembles

class SetDesc(ctypes.Structure):
    """cs_set_desc: one causal set of a batch."""
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("n", ctypes.c_int64),
                ("seed", ctypes.c_uint64)]


def _desc_array(sets):
    return (SetDesc * len(sets))(*[SetDesc(int(k), 0, int(n), int(sd)) for k, n, sd in sets])


class Batch:
    """A planned batched ensemble (cs_batch_create / cs_batch_launch).

    sets: sequence of (kind, n, seed).  The device workspace, the batch
    histogram (set s at hist_offsets[s]), actions (n_sets x n_eps) and brackets
    are torch tensors owned by this object.  launch() enqueues kernels and
    memsets only, so it can be captured into a CUDA graph.
    """

    def __init__(self, sets, path=PATH_AUTO, n_eps=4, device="cuda", stream=None):
        import torch
        self.sets = [(int(k), int(n), int(sd)) for k, n, sd in sets]
        L = lib()
        arr = _desc_array(self.sets)
        self._arr = arr
        ws = L.cs_batch_workspace_bytes(arr, len(arr), path)
        if ws == 0:
            raise CsError(-1, "cs_batch_workspace_bytes")
        self.workspace = torch.empty(ws + 1024, dtype=torch.uint8, device=device)
        base = self.workspace.data_ptr()
        self.ws_ptr = (base + 1023) // 1024 * 1024
        self.ws_bytes = ws
        h = ctypes.c_void_p()
        _check(L.cs_batch_create(arr, len(arr), path, self.ws_ptr, ws, ctypes.byref(h), _stream(stream)),
               "cs_batch_create")
        self._h = h
        self.path = L.cs_batch_path(h)
        lens = [hist_len(n) for _, n, _ in self.sets]
        self.hist_offsets = [0]
        for x in lens[:-1]:
            self.hist_offsets.append(self.hist_offsets[-1] + x)
        self.hist = torch.empty(sum(lens), dtype=torch.int64, device=device)
        self.n_eps = n_eps
        self.actions = torch.empty((len(self.sets), max(n_eps, 1)), dtype=torch.float64, device=device)
        self.brackets = torch.empty(len(self.sets), dtype=torch.int64, device=device)

    def launch(self, eps=(0.0, 0.05, 0.1, 0.2), stream=None):
        if len(eps) != self.n_eps:
            raise ValueError("eps must have n_eps entries")
        arr = (ctypes.c_double * max(len(eps), 1))(*([float(e) for e in eps] or [0.0]))
        _check(lib().cs_batch_launch(self._h, ctypes.cast(arr, ctypes.c_void_p), len(eps), self.hist.data_ptr(),
                                     self.actions.data_ptr() if eps else None, self.brackets.data_ptr(),
                                     _stream(stream)), "cs_batch_launch")

    def set_hist(self, s):
        n = self.sets[s][1]
        return self.hist[self.hist_offsets[s]:self.hist_offsets[s] + hist_len(n)]

    def status(self, stream=None) -> int:
        return lib().cs_workspace_status(self.ws_ptr, _stream(stream))

    def poll(self) -> int:
        """cs_batch_poll: PENDING (1) while the last launch runs, then its status (0 = ok); never waits."""
        return lib().cs_batch_poll(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.cs_batch_destroy(h)
            self._h = None


# ----------------------------------------------- counting slices of many sets

class CountJob(ctypes.Structure):
    """cs_count_job: one slice [item_begin, item_end) of one set's interval count."""
    _fields_ = [("bits", ctypes.c_void_p), ("n", ctypes.c_int64), ("row_words", ctypes.c_int64),
                ("hist", ctypes.c_void_p), ("operands", ctypes.c_void_p), ("item_begin", ctypes.c_int64),
                ("item_end", ctypes.c_int64)]


def count_items(n: int, path: int = PATH_AUTO) -> int:
    return lib().cs_count_items(n, path)


def peak_probe(path: int, reps: int, workspace=None) -> float:
    """cs_peak_probe: device-wide rate of the path's innermost operation
    (POPC: popc32/s; MMA: FP8 FLOP/s; MMA4: FP4 FLOP/s)."""
    import torch
    ws = workspace if workspace is not None else torch.zeros(256, dtype=torch.uint8, device="cuda")
    out = ctypes.c_double(0.0)
    _check(lib().cs_peak_probe(path, reps, _ptr(ws), ctypes.byref(out)), "cs_peak_probe")
    return out.value


def operands_bytes(n: int, path: int = PATH_MMA) -> int:
    return lib().cs_operands_bytes(n, path)


def prepare_operands(n, bits, operands_ptr, operands_nbytes, stream=None, path=PATH_MMA):
    """cs_prepare_operands: tensor-core operands of one set for `path` (operands_ptr 1024-byte aligned)."""
    _check(lib().cs_prepare_operands(n, path, _ptr(bits), bits.shape[-1], operands_ptr, operands_nbytes,
                                     _stream(stream)), "cs_prepare_operands")


def count_jobs(jobs, path, table_host_ptr, workspace_ptr, workspace_nbytes, stream=None):
    """cs_count_jobs over a sequence of CountJob (table_host_ptr: pinned, 128-byte aligned)."""
    arr = (CountJob * len(jobs))(*jobs)
    _check(lib().cs_count_jobs(arr, len(jobs), path, table_host_ptr, workspace_ptr, workspace_nbytes,
                               _stream(stream)), "cs_count_jobs")


# ------------------------------------------- degrees and sparse lists

def degrees(n, bits, kin, kout, stream=None):
    """cs_degrees: past (kin) and future (kout) relation counts, int32 tensors (either may be None)."""
    _check(lib().cs_degrees(n, _ptr(bits), bits.shape[-1], _ptr(kin), _ptr(kout), _stream(stream)), "cs_degrees")


def sparse_relations(n, bits, direction, stream=None):
    """Past (0) or future (1) sparse relation lists: (offsets int64[n+1], cols int32) device tensors.
    Synchronises once to size the column array."""
    import torch
    L = lib()
    ws = torch.empty(L.cs_sparse_workspace_bytes(n), dtype=torch.uint8, device=bits.device)
    offsets = torch.empty(n + 1, dtype=torch.int64, device=bits.device)
    _check(L.cs_sparse_offsets(n, _ptr(bits), bits.shape[-1], direction, _ptr(offsets), _ptr(ws), ws.numel(),
                               _stream(stream)), "cs_sparse_offsets")
    total = int(offsets[n].item())
    cols = torch.empty(max(total, 1), dtype=torch.int32, device=bits.device)
    _check(L.cs_sparse_columns(n, _ptr(bits), bits.shape[-1], direction, _ptr(offsets), _ptr(cols), total,
                               _ptr(ws), ws.numel(), _stream(stream)), "cs_sparse_columns")
    st = workspace_status(ws, stream)
    if st != 0:
        raise CsError(st, "cs_sparse_columns")
    return offsets, cols[:total]


# ------------------------------------------------ chains and antichains

def _chain_ws(n, device):
    import torch
    return torch.empty(lib().cs_chain_workspace_bytes(n), dtype=torch.uint8, device=device)


def longest_chain(n, bits, i=-1, j=-1, stream=None):
    """cs_longest_chain: relations on the longest chain from i to j (-1 if unrelated);
    i = j = -1: the height of the whole set in elements."""
    ws = _chain_ws(n, bits.device)
    out = ctypes.c_int64(0)
    _check(lib().cs_longest_chain(n, _ptr(bits), bits.shape[-1], i, j, ctypes.byref(out), _ptr(ws), ws.numel(),
                                  _stream(stream)), "cs_longest_chain")
    return out.value


def greedy_antichain(n, bits, seed, stream=None):
    """cs_greedy_antichain: (size, member bitset as an int64 device tensor of row_words words)."""
    import torch
    ws = _chain_ws(n, bits.device)
    members = torch.empty(bits.shape[-1], dtype=torch.int64, device=bits.device)
    out = ctypes.c_int64(0)
    _check(lib().cs_greedy_antichain(n, _ptr(bits), bits.shape[-1], seed, _ptr(members), ctypes.byref(out),
                                     _ptr(ws), ws.numel(), _stream(stream)), "cs_greedy_antichain")
    return out.value, members


# ------------------------------------------------------ failure detection

def selftest_wait(workspace, limit_s, complete=False, stream=None):
    """cs_selftest_wait: a bounded mbarrier wait that times out unless `complete`;
    read the outcome with workspace_status()."""
    _check(lib().cs_selftest_wait(_ptr(workspace), float(limit_s), 1 if complete else 0, _stream(stream)),
           "cs_selftest_wait")


def inject_fault(where, count=1):
    """cs_inject_fault: make the next `count` runs of step `where` (FAULT_*) fail; count=0 clears."""
    _check(lib().cs_inject_fault(where, count), "cs_inject_fault")
