"""ctypes binding of libftvote.so (the C ABI of include/ftvote.h).

The functions ``ft_vote``, ``ft_digest``, ``ft_plan_create``, ``ft_vote_batched``,
``ft_server_create``, ``ft_submit``, ``ft_poll`` ... have the names of the C entry
points and only marshal arguments: every step of the vote runs in the library's
CUDA kernels.  Torch is used for device memory and streams only; the helpers
``vote()``, ``digest()`` and ``Stats`` wrap the raw calls for torch tensors.

Importing this module loads the library and raises ImportError if it has not
been built (``python -m paper_1405_2912_b300.build``); there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libftvote.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1405_2912_b300.build`")
_lib = ctypes.CDLL(LIB_PATH)

FT_OK, FT_EINVAL, FT_ENOMEM, FT_EAGAIN, FT_ETIMEDOUT, FT_ECUDA, FT_ENOTFOUND = 0, -1, -2, -3, -4, -5, -6
FT_MAX_R = 8
FT_BLOCK_BYTES = 4096
DTYPE = {"i32": 0, "u32": 1, "i64": 2, "u64": 3, "u8": 4, "f32": 5, "f64": 6}
ITEMSIZE = {"i32": 4, "u32": 4, "i64": 8, "u64": 8, "u8": 1, "f32": 4, "f64": 8}


class FtError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib.ft_strerror(code).decode()
        if code == FT_ECUDA:
            msg += f" (cudaError {_lib.ft_last_cuda_error()})"
        super().__init__(f"{where}: {msg} ({code})")


class ft_stats(ctypes.Structure):
    _fields_ = [("mismatch", ctypes.c_uint64 * FT_MAX_R),
                ("first_mismatch", ctypes.c_int64 * FT_MAX_R),
                ("no_majority", ctypes.c_uint64),
                ("first_no_majority", ctypes.c_int64)]


class ft_vote_desc(ctypes.Structure):
    _fields_ = [("replicas", ctypes.c_void_p * FT_MAX_R),
                ("R", ctypes.c_int32),
                ("dtype", ctypes.c_int32),
                ("n", ctypes.c_uint64),
                ("abs_tol", ctypes.c_double),
                ("rel_tol", ctypes.c_double),
                ("out", ctypes.c_void_p),
                ("block_crc", ctypes.c_void_p),
                ("stats", ctypes.c_void_p)]


class ft_tune(ctypes.Structure):
    _fields_ = [("tile_blocks", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("warps", ctypes.c_int32),
                ("l2_prefetch", ctypes.c_int32), ("kernels", ctypes.c_int32)]


class ft_plan_group(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("R", ctypes.c_int32), ("tasks", ctypes.c_int32),
                ("warps", ctypes.c_int32), ("l2_prefetch", ctypes.c_int32), ("tile_blocks", ctypes.c_int32),
                ("tiles", ctypes.c_uint64)]


class ft_server_config(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_uint64),
                ("max_slots", ctypes.c_int32),
                ("streams", ctypes.c_int32),
                ("tile_blocks", ctypes.c_int32),
                ("max_inflight", ctypes.c_int32),
                ("max_batch_bytes", ctypes.c_uint64),
                ("reserved_sms", ctypes.c_int32),
                ("idle_spin_us", ctypes.c_int32),
                ("size_ratio", ctypes.c_int32),
                ("resident", ctypes.c_int32)]


class ft_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32),
                ("R", ctypes.c_int32),
                ("n", ctypes.c_uint64),
                ("stats", ft_stats),
                ("submit_us", ctypes.c_double),
                ("done_us", ctypes.c_double),
                ("launch_us", ctypes.c_double),
                ("launched_us", ctypes.c_double)]


class ft_unit_rating(ctypes.Structure):
    _fields_ = [("runtime", ctypes.c_double), ("valid_runs", ctypes.c_uint64), ("total_runs", ctypes.c_uint64)]


class ft_server_stats(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_uint64), ("requests", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("max_batches_in_flight", ctypes.c_int32), ("inflight_requests", ctypes.c_int32),
                ("inflight_bytes", ctypes.c_uint64), ("launch_host_us", ctypes.c_double),
                ("batch_span_us", ctypes.c_double), ("queue_us", ctypes.c_double)]


assert ctypes.sizeof(ft_stats) == 144
assert ctypes.sizeof(ft_plan_group) == 32
assert ctypes.sizeof(ft_vote_desc) == 8 * FT_MAX_R + 8 + 8 + 16 + 24

_P = ctypes.c_void_p


def _sig(name, res, *args):
    f = getattr(_lib, name, None)
    if f is None:
        return None
    f.restype = res
    f.argtypes = list(args)
    return f


ft_vote = _sig("ft_vote", ctypes.c_int, ctypes.POINTER(ft_vote_desc), _P)
ft_digest = _sig("ft_digest", ctypes.c_int, _P, ctypes.c_uint64, ctypes.c_uint32, _P, _P)
ft_plan_create = _sig("ft_plan_create", ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(ft_vote_desc),
                      ctypes.c_int32, ctypes.POINTER(ft_tune))
ft_vote_batched = _sig("ft_vote_batched", ctypes.c_int, _P, _P)
ft_vote_batched_nograph = _sig("ft_vote_batched_nograph", ctypes.c_int, _P, _P)
ft_plan_tune = _sig("ft_plan_tune", ctypes.c_int, _P, ctypes.POINTER(ft_tune))
ft_plan_destroy = _sig("ft_plan_destroy", ctypes.c_int, _P)
ft_plan_groups = _sig("ft_plan_groups", ctypes.c_int, _P, ctypes.POINTER(ft_plan_group), ctypes.c_int32,
                      ctypes.POINTER(ctypes.c_int32))
ft_server_create = _sig("ft_server_create", ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(ft_server_config))
ft_submit = _sig("ft_submit", ctypes.c_int, _P, ctypes.POINTER(ft_vote_desc), ctypes.POINTER(ctypes.c_uint64))
ft_poll = _sig("ft_poll", ctypes.c_int, _P, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ft_result))
# bulk forms: arrays are passed by address (int) so that callers can pass
# offsets into one long array without building new ctypes objects
ft_submit_many = _sig("ft_submit_many", ctypes.c_int, _P, _P, ctypes.c_int32, _P, ctypes.POINTER(ctypes.c_int32))
ft_poll_many = _sig("ft_poll_many", ctypes.c_int, _P, _P, ctypes.c_int32, ctypes.c_int64, _P,
                    ctypes.POINTER(ctypes.c_int32))
ft_server_destroy = _sig("ft_server_destroy", ctypes.c_int, _P)
ft_server_pause = _sig("ft_server_pause", ctypes.c_int, _P, ctypes.c_int32)
ft_clock_us = _sig("ft_clock_us", ctypes.c_double)
ft_server_info = _sig("ft_server_info", ctypes.c_int, _P, ctypes.POINTER(ft_server_stats))
ft_vote_host = _sig("ft_vote_host", ctypes.c_int, ctypes.POINTER(ft_vote_desc), ctypes.c_uint64)
ft_vote_many = _sig("ft_vote_many", ctypes.c_int, ctypes.POINTER(ft_vote_desc), ctypes.c_int32, _P)
ft_vote_batched_noalloc = _sig("ft_vote_batched_noalloc", ctypes.c_int, ctypes.POINTER(ft_vote_desc),
                               ctypes.c_int32, ctypes.c_int32, _P)
FT_NOALLOC_MAX_TASKS = 4096
ft_fault_probability = _sig("ft_fault_probability", ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64)
ft_fault_aware_runtime = _sig("ft_fault_aware_runtime", ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                              ctypes.c_uint64)
ft_rating_record = _sig("ft_rating_record", ctypes.c_int, ctypes.POINTER(ft_unit_rating), ctypes.c_int32,
                        ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, ctypes.POINTER(ft_stats))
ft_rating_rank = _sig("ft_rating_rank", ctypes.c_int, ctypes.POINTER(ft_unit_rating), ctypes.c_int32,
                      ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32),
                      ctypes.POINTER(ctypes.c_int32))
ft_ckpt_create = _sig("ft_ckpt_create", ctypes.c_int, ctypes.POINTER(_P), ctypes.c_uint64, ctypes.c_uint64)
ft_ckpt_sync = _sig("ft_ckpt_sync", ctypes.c_int, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_uint64))
ft_ckpt_restore = _sig("ft_ckpt_restore", ctypes.c_int, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_uint64))
ft_ckpt_destroy = _sig("ft_ckpt_destroy", ctypes.c_int, _P)
ft_ckpt_forget = _sig("ft_ckpt_forget", ctypes.c_int, _P)
FT_MEM_HOST, FT_MEM_DEVICE, FT_ACCESS_READ, FT_ACCESS_WRITE = 0, 1, 1, 2
ft_area_create = _sig("ft_area_create", ctypes.c_int, ctypes.POINTER(_P), _P, ctypes.c_uint64)
ft_area_request = _sig("ft_area_request", ctypes.c_int, _P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_P), _P,
                       ctypes.POINTER(ctypes.c_uint64))
ft_area_invalidate = _sig("ft_area_invalidate", ctypes.c_int, _P, ctypes.c_int32)
ft_area_versions = _sig("ft_area_versions", ctypes.c_int, _P, ctypes.POINTER(ctypes.c_uint64),
                        ctypes.POINTER(ctypes.c_uint64))
ft_area_destroy = _sig("ft_area_destroy", ctypes.c_int, _P)
FT_PAPER_F32_REL_TOL = 1e-3
ft_register_data = _sig("ft_register_data", ctypes.c_int, _P, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double,
                        ctypes.c_double)
ft_unregister_data = _sig("ft_unregister_data", ctypes.c_int, _P)
ft_registered_type = _sig("ft_registered_type", ctypes.c_int, _P, ctypes.POINTER(ctypes.c_int32),
                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_uint64))
ft_vote_registered = _sig("ft_vote_registered", ctypes.c_int, ctypes.POINTER(_P), ctypes.c_int32, _P, _P, _P, _P)
ft_task_fn = ctypes.CFUNCTYPE(ctypes.c_int, _P, ctypes.c_int32, _P, _P)
ft_dmr_run = _sig("ft_dmr_run", ctypes.c_int, ft_task_fn, _P, ctypes.POINTER(ft_vote_desc), _P)
ft_strerror = _sig("ft_strerror", ctypes.c_char_p, ctypes.c_int)
ft_last_cuda_error = _sig("ft_last_cuda_error", ctypes.c_int)
ft_launch_count = _sig("ft_launch_count", ctypes.c_uint64)
ft_version = _sig("ft_version", ctypes.c_char_p)


def check(code: int, where: str) -> int:
    if code != FT_OK:
        raise FtError(code, where)
    return code


# ---------------------------------------------------------------------------
# torch helpers (argument marshalling only)
# ---------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def dtype_name(t) -> str:
    torch = _torch()
    m = {torch.float32: "f32", torch.float64: "f64", torch.int32: "i32", torch.int64: "i64",
         torch.uint8: "u8"}
    for name in ("uint32", "uint64"):
        if hasattr(torch, name):
            m[getattr(torch, name)] = "u" + name[4:]
    if t not in m:
        raise TypeError(f"unsupported element type {t}")
    return m[t]


def stream_handle(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def new_stats(device="cuda"):
    """A device buffer holding one ft_stats (18 x 8 bytes)."""
    torch = _torch()
    return torch.empty(18, dtype=torch.int64, device=device)


def parse_stats(buf, R: int) -> dict:
    """Host dict from an ft_stats buffer (a torch tensor of 18 int64 or bytes)."""
    v = buf.cpu().tolist() if hasattr(buf, "cpu") else list(buf)
    mism = [x & 0xFFFFFFFFFFFFFFFF for x in v[0:R]]
    return {"mismatch": mism, "first_mismatch": v[8:8 + R], "no_majority": v[16] & 0xFFFFFFFFFFFFFFFF,
            "first_no_majority": v[17]}


def make_desc(replicas, out, block_crc, stats, abs_tol=0.0, rel_tol=0.0, dtype=None, n=None) -> ft_vote_desc:
    """Descriptor from torch tensors (or raw device addresses with dtype and n)."""
    d = ft_vote_desc()
    R = len(replicas)
    ptrs = [r if isinstance(r, int) else r.data_ptr() for r in replicas]
    for i, p in enumerate(ptrs[:FT_MAX_R]):
        d.replicas[i] = p
    d.R = R
    if dtype is None:
        dtype = dtype_name(replicas[0].dtype)
    d.dtype = DTYPE[dtype] if isinstance(dtype, str) else int(dtype)
    d.n = n if n is not None else replicas[0].numel()
    d.abs_tol = float(abs_tol)
    d.rel_tol = float(rel_tol)
    d.out = out if isinstance(out, int) or out is None else out.data_ptr()
    d.block_crc = block_crc if isinstance(block_crc, int) or block_crc is None else block_crc.data_ptr()
    d.stats = stats if isinstance(stats, int) or stats is None else stats.data_ptr()
    return d


def n_blocks(nbytes: int, block_bytes: int = FT_BLOCK_BYTES) -> int:
    return (nbytes + block_bytes - 1) // block_bytes


def vote(replicas, abs_tol=0.0, rel_tol=0.0, out=None, block_crc=None, stats=None, stream=None,
         with_crc=True):
    """ft_vote on torch CUDA tensors.  Returns (out, block_crc, stats buffer)."""
    torch = _torch()
    x0 = replicas[0]
    if out is None:
        out = torch.empty_like(x0)
    if block_crc is None and with_crc:
        block_crc = torch.empty(n_blocks(x0.numel() * x0.element_size()), dtype=torch.int32, device=x0.device)
    if stats is None:
        stats = new_stats(x0.device)
    d = make_desc(replicas, out, block_crc, stats, abs_tol, rel_tol)
    check(ft_vote(ctypes.byref(d), stream_handle(stream)), "ft_vote")
    return out, block_crc, stats


def digest(buf, block_bytes=FT_BLOCK_BYTES, out=None, stream=None):
    """ft_digest of a torch CUDA tensor's bytes.  Returns an int32 tensor of CRCs."""
    torch = _torch()
    nbytes = buf.numel() * buf.element_size()
    if out is None:
        out = torch.empty(max(1, n_blocks(nbytes, block_bytes)), dtype=torch.int32, device=buf.device)
    check(ft_digest(buf.data_ptr(), nbytes, block_bytes, out.data_ptr(), stream_handle(stream)), "ft_digest")
    return out
