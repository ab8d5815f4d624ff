"""ctypes signatures of every function in include/ising.h."""
from __future__ import annotations

import ctypes


class IsingJob(ctypes.Structure):
    """struct ising_job (include/ising.h)."""
    _fields_ = [("L", ctypes.c_int32), ("beta", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("hot", ctypes.c_int32), ("sweeps", ctypes.c_int64), ("every", ctypes.c_int64),
                ("host_E", ctypes.POINTER(ctypes.c_int64)), ("host_M", ctypes.POINTER(ctypes.c_int64)),
                ("host_spins", ctypes.POINTER(ctypes.c_int8)), ("rng", ctypes.c_int32)]


class IsingResult(ctypes.Structure):
    """struct ising_result (include/ising.h)."""
    _fields_ = [("status", ctypes.c_int32), ("state", ctypes.c_int32), ("submit_s", ctypes.c_double),
                ("start_s", ctypes.c_double), ("done_s", ctypes.c_double), ("sweeps_done", ctypes.c_int64)]

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_sz = ctypes.c_size_t
_int = ctypes.c_int
_dbl = ctypes.c_double
_cstr = ctypes.c_char_p
_pi64 = ctypes.POINTER(ctypes.c_int64)
_pu64 = ctypes.POINTER(ctypes.c_uint64)
_pi32 = ctypes.POINTER(ctypes.c_int32)
_pu32 = ctypes.POINTER(ctypes.c_uint32)
_pi8 = ctypes.POINTER(ctypes.c_int8)
_pu8 = ctypes.POINTER(ctypes.c_uint8)
_pd = ctypes.POINTER(ctypes.c_double)
_pvp = ctypes.POINTER(ctypes.c_void_p)

SYMBOLS = {
    "ising_strerror": (_cstr, [_int]),
    "ising_last_cuda_error": (_cstr, []),
    "ising_bytes_required": (_sz, [_i32]),
    "ising_create": (_int, [_i32, _u64, _pvp]),
    "ising_create_on": (_int, [_i32, _u64, _vp, _sz, _vp, _pvp]),
    "ising_create_layout": (_int, [_i32, _u64, _i32, _pvp]),
    "ising_destroy": (_int, [_vp]),
    "ising_init_hot": (_int, [_vp]),
    "ising_init_cold": (_int, [_vp, ctypes.c_int8]),
    "ising_set_beta": (_int, [_vp, _dbl]),
    "ising_get_thresholds": (_int, [_vp, _pu64]),
    "ising_sweep": (_int, [_vp, _i64]),
    "ising_sweep_record": (_int, [_vp, _i64, _i64, _pi64, _pi64]),
    "ising_energy": (_int, [_vp, _pi64]),
    "ising_magnetization": (_int, [_vp, _pi64]),
    "ising_means": (_int, [_pi64, _pi64, _i64, _i32, _pd, _pd]),
    "ising_get_spins": (_int, [_vp, _pi8, _sz]),
    "ising_set_spins": (_int, [_vp, _pi8, _sz]),
    "ising_get_words": (_int, [_vp, _pu64, _sz]),
    "ising_set_words": (_int, [_vp, _pu64, _sz]),
    "ising_layout": (_int, [_vp, _pi32, _pi32, _pi32]),
    "ising_get_sweep": (_int, [_vp, _pu64]),
    "ising_set_sweep": (_int, [_vp, _u64]),
    "ising_set_stream": (_int, [_vp, _vp]),
    "ising_set_item_lanes": (_int, [_vp, _i32]),
    "ising_run_states": (_int, [_vp, _vp, _i32, _i64, _i64, _vp, _vp]),
    "ising_set_tiling": (_int, [_vp, _i32, _i32, _i32]),
    "ising_device_words": (_int, [_vp, _i32, _pvp]),
    "ising_set_path": (_int, [_vp, _i32]),
    "ising_get_path": (_int, [_vp, _vp]),
    "ising_set_clusters": (_int, [_vp, _i32]),
    "ising_cluster_inject_stall": (_int, [_vp, _i32]),
    "ising_cluster_inject_absent": (_int, [_vp, _i32]),
    "ising_set_rng": (_int, [_vp, _i32]),
    "ising_set_chain": (_int, [_vp, _i32, _i32]),
    "ising_philox_blocks": (_int, [_u64, _pu32, _pu32, _i64]),
    "ising_batch_create": (_int, [_i32, _pi32, _pd, _pu64, _pu8, _pvp]),
    "ising_batch_destroy": (_int, [_vp]),
    "ising_batch_sweep": (_int, [_vp, _pi64, _i64, _vp, _vp]),
    "ising_batch_get_spins": (_int, [_vp, _i32, _pi8, _sz]),
    "ising_batch_get_sweep": (_int, [_vp, _i32, _pu64]),
    "ising_batch_set_tiling": (_int, [_vp, _i32, _i32]),
    "ising_batch_set_rng": (_int, [_vp, _i32]),
    "ising_batch_set_lanes": (_int, [_vp, _i32]),
    "ising_batch_run": (_int, [_i32, _pi32, _pd, _pu64, _pu8, _pi64, _i64, _vp, _vp, _vp]),
    "ising_server_create": (_int, [_sz, _pvp]),
    "ising_server_create_ex": (_int, [_sz, _i32, _i32, _pvp]),
    "ising_server_inject_fault": (_int, [_vp, _i32]),
    "ising_server_submit": (_int, [_vp, ctypes.POINTER(IsingJob), _pu64]),
    "ising_server_poll": (_int, [_vp, _u64, ctypes.POINTER(IsingResult)]),
    "ising_server_wait": (_int, [_vp, _u64, _i64, ctypes.POINTER(IsingResult)]),
    "ising_server_cancel": (_int, [_vp, _u64]),
    "ising_server_release": (_int, [_vp, _u64]),
    "ising_server_stats": (_int, [_vp, _pi64, _pd, _pi64, _pd]),
    "ising_server_destroy": (_int, [_vp]),
    "ising_autotune": (_int, [_i32, _i32, _pi32, _pi32, _pi32, _pi32, _pd]),
    "ising_probe_int_pipes": (_int, [_pd, _pd, _pd, _pi32]),
    "ising_check_status": (_int, [_pi32, _pu64]),
    "ising_batch_autotune": (_int, [_i32, _pi32, _pd, _pu64, _pu8, _i64, _i64, _pi32, _pi32, _pi32, _pd]),
    "ising_sweep_record_noalloc": (_int, [_vp, _vp, _i32, _u64, _dbl, _u64, _i64, _i64, _pi64, _pi64, _vp]),
}


def declare(lib: ctypes.CDLL) -> None:
    for name, (res, args) in SYMBOLS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
