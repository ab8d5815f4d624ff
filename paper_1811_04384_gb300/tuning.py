"""Autotuned launch shapes (ising_autotune / ising_batch_autotune in
include/ising.h), kept in a JSON table next to this file:

    {"device": "...", "lattice": {"<L>": {"block_words": .., "block_groups": ..,
     "path": .., "item_lanes": .., "ns_per_update": ..}},
     "batch": {"<name>": {"threads_per_tile": .., "graph_chunk": .., "lanes": ..,
     "ns_per_update": .., "workload": ".."}}}

`apply(lattice)` sets the tuned shape for the lattice's side and
`apply_batch(batch, name)` the tuned tiles of a named batch workload, when the
table holds one for the current device.  Choosing a shape never changes
results.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

from . import _check, load

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def _device_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:
        return "unknown"


def tune_lattice(L: int, sweeps: int = 20) -> dict:
    bw, bg, path, lanes = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    ns = ctypes.c_double()
    _check(load().ising_autotune(int(L), int(sweeps), ctypes.byref(bw), ctypes.byref(bg), ctypes.byref(path),
                                 ctypes.byref(lanes), ctypes.byref(ns)), "ising_autotune")
    return {"block_words": bw.value, "block_groups": bg.value, "path": path.value, "item_lanes": lanes.value,
            "ns_per_update": ns.value}


def tune_batch(L, beta, seed, hot, sweeps: int = 50, every: int = 1) -> dict:
    L = np.ascontiguousarray(L, dtype=np.int32)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    seed = np.ascontiguousarray(seed, dtype=np.uint64)
    hot = np.ascontiguousarray(hot, dtype=np.uint8)
    th, ch, ln = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    ns = ctypes.c_double()
    _check(load().ising_batch_autotune(len(L), L.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                       beta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       seed.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                       hot.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), int(sweeps), int(every),
                                       ctypes.byref(th), ctypes.byref(ch), ctypes.byref(ln), ctypes.byref(ns)),
           "ising_batch_autotune")
    return {"threads_per_tile": th.value, "graph_chunk": ch.value, "lanes": ln.value, "ns_per_update": ns.value}


def load_table(path: str = TABLE) -> dict:
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def save_table(table: dict, path: str = TABLE):
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


def tune_all(Ls, sweeps: int = 20, path: str = TABLE) -> dict:
    table = load_table(path)
    if table.get("device") != _device_name():
        table = {}
    table["device"] = _device_name()
    table["lattice"] = {}
    for L in Ls:
        table["lattice"][str(int(L))] = tune_lattice(int(L), sweeps)
    save_table(table, path)
    return table


def tune_named_batch(name: str, L, beta, seed, hot, sweeps: int = 20, every: int = 1, workload: str = "",
                     path: str = TABLE) -> dict:
    """Tune the batch tiles of one workload and store them under `name`."""
    entry = tune_batch(L, beta, seed, hot, sweeps, every)
    entry["workload"] = workload
    table = load_table(path)
    if table.get("device") != _device_name():
        table = {"lattice": {}}
    table["device"] = _device_name()
    table.setdefault("batch", {})[name] = entry
    save_table(table, path)
    return entry


def apply_batch(batch, name: str, table: dict | None = None) -> bool:
    """Set the tuned tiles of batch workload `name` if the table has them for
    this device."""
    table = load_table() if table is None else table
    entry = table.get("batch", {}).get(name)
    if not entry or table.get("device") != _device_name():
        return False
    batch.set_tiling(entry["threads_per_tile"], entry["graph_chunk"])
    batch.set_lanes(entry["lanes"])
    return True


def apply(lattice, table: dict | None = None) -> bool:
    """Set the tuned tiling/path of lattice.L if the table has one for this device."""
    table = load_table() if table is None else table
    entry = table.get("lattice", {}).get(str(lattice.L))
    if not entry or table.get("device") != _device_name():
        return False
    lattice.set_path(entry["path"])
    if entry["path"] == 1:
        lattice.set_tiling(4, entry["block_words"], entry["block_groups"])
        lattice.set_item_lanes(entry.get("item_lanes", 0))
    return True
