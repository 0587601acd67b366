"""Helpers shared by the GPU parity tests: encode oracle trees in the packed node format that
include/aiwcrf.h documents, and compare them with a serialized GPU forest."""
from __future__ import annotations

import numpy as np

LEAF = np.uint64(1 << 63)
MASK63 = np.uint64((1 << 63) - 1)


def encode_oracle_tree(tr) -> np.ndarray:
    """Packed u64 nodes of an oracle tree (the documented encoding, written independently)."""
    out = np.zeros(tr.num_nodes, np.uint64)
    for j in range(tr.num_nodes):
        if tr.feature[j] < 0:
            out[j] = LEAF | (np.int64(tr.value[j]).view(np.uint64) & MASK63)
        else:
            thr = int(np.float32(tr.thr[j]).view(np.uint32))
            out[j] = np.uint64((int(tr.feature[j]) << 56) | (int(tr.left[j]) << 32) | thr)
    return out


def gpu_tree(dec: dict, t: int) -> np.ndarray:
    off = dec["tree_off"]
    return dec["nodes"][off[t]:off[t + 1]]


def assert_tree_equal(gpu_nodes: np.ndarray, oracle_tree, where: str = ""):
    exp = encode_oracle_tree(oracle_tree)
    m = exp.size
    assert gpu_nodes.size in (m, m + 1), f"{where}: {gpu_nodes.size} packed nodes, oracle has {m}"
    if gpu_nodes.size == m + 1:
        assert gpu_nodes[m] == LEAF, f"{where}: padding node is not the zero leaf"
    bad = np.flatnonzero(gpu_nodes[:m] != exp)
    assert bad.size == 0, (f"{where}: {bad.size} nodes differ, first at {bad[0]}: "
                           f"gpu {int(gpu_nodes[bad[0]]):#018x} oracle {int(exp[bad[0]]):#018x}")


def walk_packed(nodes: np.ndarray, x: np.ndarray) -> int:
    """Leaf value reached by one query in one packed tree (reference walk for large checks)."""
    j = 0
    while True:
        nd = int(nodes[j])
        if nd >> 63:
            v = nd & ((1 << 63) - 1)
            return v - (1 << 63) if v >> 62 else v
        f = (nd >> 56) & 0x7F
        lc = (nd >> 32) & 0xFFFFFF
        thr = np.uint32(nd & 0xFFFFFFFF).view(np.float32)
        j = lc + (0 if x[f] <= thr else 1)
