"""ctypes binding of libbbtn.so (argument marshalling only; all compute is in the library).

The functions mirror include/bbtn.h one to one. Device buffers are passed as raw
pointers (e.g. ``tensor.data_ptr()`` of CUDA tensors), streams as ``int`` handles
(``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbbtn.so")

OK, EINVAL, ENOMEM, EOVERFLOW, ETIMEOUT, EIO, ECUDA, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
NEG = -(1 << 29)
FINITE_MIN = -(1 << 28)
MAX_PRIMES = 8
MODE_PLAIN, MODE_SLICED, MODE_BBTN = 0, 1, 2


class BBTNError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bbtn error {code}: {msg}")
        self.code = code


class Opts(C.Structure):
    _fields_ = [("space_cap_log2", C.c_int), ("n_primes", C.c_int), ("seed", C.c_uint64),
                ("mode", C.c_int), ("sa_iters", C.c_int), ("region_size", C.c_int),
                ("batch", C.c_int), ("use_gnn", C.c_int), ("count_check", C.c_int),
                ("use_symmetry", C.c_int), ("verbose", C.c_int), ("profile", C.c_int),
                ("max_slices_log2", C.c_int), ("branch_lookahead", C.c_int), ("leaf_trials", C.c_int),
                ("autotune", C.c_int), ("wide_counts", C.c_int), ("slice_sample", C.c_int), ("arena_budget_mb", C.c_int), ("no_chain_fusion", C.c_int),
                ("order_restarts", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("t_total_s", C.c_double), ("t_plan_s", C.c_double), ("t_device_s", C.c_double),
                ("tropical_ops", C.c_double), ("bytes_moved", C.c_double), ("kernel_ms", C.c_double),
                ("nodes", C.c_int64), ("leaves", C.c_int64), ("pruned", C.c_int64),
                ("launches", C.c_int64), ("steps", C.c_int64), ("sc_log2", C.c_int),
                ("tc_log2", C.c_double), ("sc_plain_log2", C.c_double), ("slices_log2", C.c_int),
                ("prof_ms", C.c_double), ("prof_bytes", C.c_double), ("prof_ops", C.c_double),
                ("prof_launches", C.c_int64), ("prof_scount_ms", C.c_double), ("prof_scount_bytes", C.c_double),
                ("prof_scount_launches", C.c_int64), ("prof_stream_ms", C.c_double),
                ("prof_stream_bytes", C.c_double), ("prof_stream_launches", C.c_int64),
                ("prof_tiled_ms", C.c_double), ("prof_tiled_ops", C.c_double), ("prof_tiled_launches", C.c_int64),
                ("prof_tiled16_launches", C.c_int64), ("prof_tcount_ms", C.c_double),
                ("prof_tcount_ops", C.c_double), ("prof_tcount_launches", C.c_int64), ("slices_run", C.c_int64),
                ("prof_chain_ms", C.c_double), ("prof_chain_bytes", C.c_double), ("prof_chain_launches", C.c_int64),
                ("chains", C.c_int64), ("chained_steps", C.c_int64), ("bwd_kept", C.c_int64),
                ("bwd_recomputed", C.c_int64), ("bwd_peak_bytes", C.c_double), ("bwd_keep_all_bytes", C.c_double),
                ("bwd_budget_bytes", C.c_double), ("prof_tiled_bytes", C.c_double),
                ("prof_tcount_bytes", C.c_double)]

    def as_dict(self):
        return {k: (getattr(self, k) if k != "reserved" else None) for k, _ in self._fields_ if k != "reserved"}


class PlanInfo(C.Structure):
    _fields_ = [("tc_log2", C.c_double), ("sc_log2", C.c_int), ("rho", C.c_double),
                ("slices_log2", C.c_int), ("steps", C.c_int64), ("ops", C.c_double), ("bytes", C.c_double),
                ("arena_bytes", C.c_double), ("bb_nodes", C.c_int64), ("bb_leaves", C.c_int64),
                ("chains", C.c_int), ("chained_steps", C.c_int), ("bwd_kept", C.c_int), ("bwd_recomputed", C.c_int),
                ("bwd_peak_bytes", C.c_double), ("bwd_keep_all_bytes", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_lib = None

_P = C.POINTER
_i32p, _u64p, _i64p, _i8p, _f32p = _P(C.c_int32), _P(C.c_uint64), _P(C.c_int64), _P(C.c_int8), _P(C.c_float)
_vp = C.c_void_p

_SIGS = {
    "bbtn_version": ([], C.c_char_p),
    "bbtn_last_error": ([], C.c_char_p),
    "bbtn_primes": ([C.c_int, _u64p], C.c_int),
    "bbtn_prime_pairs": ([C.c_int, _u64p], C.c_int),
    "bbtn_crt_decimal": ([C.c_int, _u64p, _u64p, C.c_char_p, C.c_size_t, _P(C.c_size_t)], C.c_int),
    "bbtn_contract": ([C.c_int, _i32p, _vp, _vp, C.c_int, _i32p, _vp, _vp, C.c_int, _i32p, _vp, _vp,
                       C.c_int, _u64p, _vp], C.c_int),
    "bbtn_contract_chain": ([C.c_int, _i32p, _vp, C.c_int, _i32p, _i32p, _P(_vp), _i32p, _i32p, _vp, _vp],
                            C.c_int),
    "bbtn_contract_values16": ([C.c_int, _i32p, _vp, C.c_int, _i32p, _vp, C.c_int, _i32p, _vp, _vp], C.c_int),
    "bbtn_permute": ([C.c_int, _i32p, _vp, _vp, _vp, _vp, C.c_int, _vp], C.c_int),
    "bbtn_permute_uses_tma": ([C.c_int, _i32p, _vp, _vp, _vp, _vp, C.c_int], C.c_int),
    "bbtn_search_leaves": ([_vp, C.c_int64, _i8p, _P(C.c_int64)], C.c_int),
    "bbtn_prepare": ([_vp], C.c_int),
    "bbtn_clear_order_cache": ([], C.c_int),
    "bbtn_aggregate": ([C.c_int64, _vp, _vp, C.c_int, _u64p, _vp, _vp, _vp], C.c_int),
    "bbtn_contract_backward": ([C.c_int, _i32p, _vp, C.c_int, _i32p, _vp, C.c_int, _i32p, _vp,
                                C.c_int64, _vp, _vp, _vp, _vp], C.c_int),
    "bbtn_default_opts": ([_P(Opts)], None),
    "bbtn_create": ([_P(Opts), _P(_vp)], C.c_int),
    "bbtn_destroy": ([_vp], None),
    "bbtn_set_stream": ([_vp, _vp], C.c_int),
    "bbtn_set_workspace": ([_vp, _vp, C.c_size_t], C.c_int),
    "bbtn_load_spin_glass": ([_vp, C.c_int, C.c_int, _i32p, _i32p, _i32p], C.c_int),
    "bbtn_load_mwis": ([_vp, C.c_int, C.c_int, _i32p, _i32p], C.c_int),
    "bbtn_load_file": ([_vp, C.c_char_p], C.c_int),
    "bbtn_solve": ([_vp, C.c_int, C.c_int], C.c_int),
    "bbtn_get_energy": ([_vp, _i64p], C.c_int),
    "bbtn_shard_values": ([_vp, C.c_int, C.c_int, C.c_int, _i64p], C.c_int),
    "bbtn_shard_counts": ([_vp, C.c_int64, C.c_int, _i32p, _u64p, _u64p, _P(C.c_int), _P(C.c_int), _i8p,
                           _P(C.c_int)], C.c_int),
    "bbtn_count_decimal": ([C.c_int, C.c_int, _u64p, _u64p, C.c_char_p, C.c_size_t, _P(C.c_size_t)], C.c_int),
    "bbtn_get_count_residues": ([_vp, _u64p, _u64p, _P(C.c_int)], C.c_int),
    "bbtn_get_count_dec": ([_vp, C.c_char_p, C.c_size_t, _P(C.c_size_t)], C.c_int),
    "bbtn_get_config": ([_vp, _i8p], C.c_int),
    "bbtn_get_stats": ([_vp, _P(Stats)], C.c_int),
    "bbtn_analyze": ([_vp, _P(PlanInfo), C.c_char_p], C.c_int),
    "bbtn_aggregate_noalloc": ([C.c_int64, _vp, _vp, C.c_int, _u64p, _vp, _vp, _vp], C.c_int),
    "bbtn_aggregate_noalloc_max_scratch": ([], C.c_size_t),
    "bbtn_bench_alu": ([C.c_int, C.c_int, C.c_int, C.c_int, _P(C.c_double), _f32p, _vp], C.c_int),
    "bbtn_gnn_create": ([C.c_uint64, _P(_vp)], C.c_int),
    "bbtn_gnn_destroy": ([_vp], None),
    "bbtn_gnn_param_count": ([], C.c_int),
    "bbtn_gnn_set_stream": ([_vp, _vp], C.c_int),
    "bbtn_gnn_features": ([C.c_int, C.c_int, _i32p, _i32p, _i8p, _f32p, _f32p], C.c_int),
    "bbtn_gnn_set_graph": ([_vp, C.c_int, C.c_int, _i32p], C.c_int),
    "bbtn_gnn_forward": ([_vp, _f32p, _f32p], C.c_int),
    "bbtn_gnn_train_step": ([_vp, _f32p, _f32p, _f32p, C.c_float, _f32p], C.c_int),
    "bbtn_gnn_get_params": ([_vp, _f32p], C.c_int),
    "bbtn_gnn_set_params": ([_vp, _f32p], C.c_int),
    "bbtn_gnn_get_grads": ([_vp, _f32p], C.c_int),
    "bbtn_set_gnn": ([_vp, _vp, _vp], C.c_int),
    "bbtn_branch_samples": ([_vp, C.c_int, C.c_int, _i8p, _f32p, _f32p, _P(C.c_int)], C.c_int),
}


def load():
    """Load libbbtn.so from the package directory; raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2602_05470_gb300.build` "
                          "(there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (args, res) in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def check(rc):
    if rc != OK:
        raise BBTNError(rc, load().bbtn_last_error().decode())
    return rc


def i32_array(seq):
    seq = [int(x) for x in seq]
    return (C.c_int32 * max(len(seq), 1))(*seq)


def u64_array(seq):
    seq = [int(x) for x in seq]
    return (C.c_uint64 * max(len(seq), 1))(*seq)
