"""The pipelined gather's per-tile re-encoding of the map (csrc/bs_tiles.h),
compiled on the host and checked without a GPU.

For each tile the encoding must give the kernel, from shared memory alone,
every entry of every row in CSR order.  The chunk ids must be sorted and
distinct, and must stay inside q_L (the last odd node's chunk never appears).
The offsets must address the staged chunk values of the right local nodes.
The row starts must match the CSR, and the summing order must be a permutation
of the tile's rows by non-increasing length.  The sizes must stay within the
kernel's stage.  Tiles marked -1 hold one row summed from the CSR: a row with
more entries or chunks than a tile holds, or the row of the last local node
when N_L is odd.  Decoding the
encoding as the kernel does and summing each row serially from +0 must give
the oracle's gather bit for bit.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2009_10917_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2009_10917_gb300", "csrc")

WRAP = r"""
#include "bs_tiles.h"
#include <cstring>
static bs::AgTiles g_t;
extern "C" {
void limits(int *out) {
  out[0] = bs::kAgChunks; out[1] = bs::kAgEntries; out[2] = bs::kAgRows; out[3] = bs::kAgBlob16;
}
void build(const int32_t *rs, int64_t ng, const int32_t *col, int64_t nnz, int64_t nl,
           int64_t *sizes) {
  std::vector<int32_t> r(rs, rs + ng + 1), c(col, col + nnz);
  g_t = bs::build_async_tiles(r, c, nl, ng);
  sizes[0] = (int64_t)g_t.info.size();
  sizes[1] = (int64_t)g_t.chunks.size();
  sizes[2] = (int64_t)g_t.blob.size();
}
void fetch(int32_t *info, int32_t *chunks, uint16_t *blob) {
  std::memcpy(info, g_t.info.data(), sizeof(bs::AgInfo) * g_t.info.size());
  std::memcpy(chunks, g_t.chunks.data(), sizeof(int32_t) * g_t.chunks.size());
  std::memcpy(blob, g_t.blob.data(), sizeof(uint16_t) * g_t.blob.size());
}
}
"""


@pytest.fixture(scope="module")
def enc(tmp_path_factory):
    d = tmp_path_factory.mktemp("tiles")
    src, so = d / "wrap.cpp", d / "wrap.so"
    src.write_text(WRAP)
    subprocess.run(["g++", "-std=c++17", "-O2", "-Wall", "-Werror", "-shared", "-fPIC", "-I", CSRC,
                    str(src), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    lim = (ctypes.c_int * 4)()
    L.limits(lim)
    return L, tuple(lim)


def encode(L, ids, NL, NG):
    rs, ci = oracle.csr(ids, NG)
    rs = np.ascontiguousarray(rs, dtype=np.int32)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    sizes = np.zeros(3, dtype=np.int64)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    L.build(p(rs), ctypes.c_int64(NG), p(ci), ctypes.c_int64(ci.size), ctypes.c_int64(NL),
            p(sizes))
    info = np.zeros((int(sizes[0]), 4), dtype=np.int32)
    chunks = np.zeros(int(sizes[1]), dtype=np.int32)
    blob = np.zeros(int(sizes[2]), dtype=np.uint16)
    L.fetch(p(info), p(chunks), p(blob))
    return rs, ci, info, chunks, blob


def pad8(n):
    return (n + 7) // 8 * 8


def decode_and_gather(lim, rs, ci, info, chunks, blob, ql, NL, NG):
    """The kernel's reading of the encoding, every invariant asserted on the
    way; returns the gathered q_G (serial sums from +0 in the encoded order)."""
    max_chunks, max_entries, max_rows, max_blob16 = lim
    qg = np.full(NG, np.nan)
    assert info[0, 0] == 0 and info[-1, 0] == NG
    for t in range(info.shape[0] - 1):
        r0, c0, b0, meta = info[t]
        r1, c1, b1 = info[t + 1, 0], info[t + 1, 1], info[t + 1, 2]
        assert r1 > r0
        if meta < 0:  # rows summed from the CSR
            assert c1 == c0 and b1 == b0
            assert r1 - r0 == 1  # a -1 tile holds one row
            lo, hi = rs[r0], rs[r0 + 1]
            too_many_entries = hi - lo > max_entries
            too_many_chunks = np.unique(ci[lo:hi] >> 1).size > max_chunks
            odd_last = NL % 2 == 1 and hi > lo and ci[hi - 1] == NL - 1
            assert too_many_entries or too_many_chunks or odd_last
            s = 0.0
            for k in range(lo, hi):
                s = (0.0 + ql[ci[k]]) if k == lo else s + ql[ci[k]]
            qg[r0] = s
            continue
        ne, rows = meta >> 16, meta & 0xFFFF
        assert rows == r1 - r0 and rows <= max_rows and ne <= max_entries
        assert ne == rs[r1] - rs[r0]
        ch = chunks[c0:c1]
        assert ch.size <= max_chunks and np.all(np.diff(ch) > 0)
        assert np.all(ch >= 0) and np.all(2 * ch + 1 < NL)  # never the odd last node's chunk
        assert b1 - b0 <= max_blob16
        words = blob[8 * b0:8 * b1]
        off = words[:ne]
        rstart = words[pad8(ne):pad8(ne) + rows + 1].astype(np.int64)
        order = words[pad8(ne) + pad8(rows + 1):pad8(ne) + pad8(rows + 1) + rows].astype(np.int64)
        assert pad8(ne) + pad8(rows + 1) + pad8(rows) == words.size
        lens = np.diff(rstart)
        assert rstart[0] == 0 and rstart[-1] == ne and np.all(lens >= 0)
        assert np.array_equal(lens, np.diff(rs[r0:r1 + 1]))
        assert np.array_equal(np.sort(order), np.arange(rows))
        assert np.all(np.diff(lens[order]) <= 0)  # longest rows first
        staged = np.empty(2 * ch.size)
        staged[0::2], staged[1::2] = ql[2 * ch], ql[2 * ch + 1]
        assert np.all(off < staged.size)
        # each entry addresses the value of its own local node
        assert np.array_equal(2 * ch[off >> 1] + (off & 1), ci[rs[r0]:rs[r1]])
        for q in order:
            a, b = rstart[q], rstart[q + 1]
            s = 0.0
            for k in range(a, b):
                s = (0.0 + staged[off[k]]) if k == a else s + staged[off[k]]
            qg[r0 + q] = s
    return qg


def bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


CASES = [(4, 3, 0.0), (3, 2, 0.0), (5, 4, 0.05), (2, 7, 0.0), (3, 5, 0.1), (7, 1, 0.0),
         (2, 15, 0.0)]


@pytest.mark.parametrize("K,N,frac", CASES)
def test_encoding_reproduces_the_gather(enc, K, N, frac):
    L, lim = enc
    m = synth.Mesh(K, N, seed=K * 11 + N)
    ids = m.ids.copy()
    if frac > 0:
        ids[synth.uniform(ids.size, 17, 0, 0.0, 1.0) < frac] = -1
    rs, ci, info, chunks, blob = encode(L, ids, m.NL, m.NG)
    ql = synth.uniform(m.NL, 18)
    ql[::37] = -0.0  # signed zeros: the sums start from +0
    got = decode_and_gather(lim, rs, ci, info, chunks, blob, ql, m.NL, m.NG)
    assert np.array_equal(bits(got), bits(oracle.gather(ids, ql, m.NG)))


def test_long_rows_and_odd_last_node(enc):
    """A row of 1500 copies (longer than a tile) and one of 900 (long but
    fitting); the last local node of an odd N_L masked, or on a row of 300
    copies; global nodes with no copies at all."""
    L, lim = enc
    m = synth.Mesh(5, 2, seed=3)  # N_L = 3375, odd
    assert m.NL % 2 == 1
    for variant in range(3):
        ids = m.ids.copy()
        if variant == 0:
            ids[:1500] = 0
            ids[2000:2900] = 9
        elif variant == 1:
            ids[-1] = -1
            ids[100:140] = -1  # some global nodes lose every copy
        else:
            ids[-300:] = 5     # the last local node on a row of 300 copies
        rs, ci, info, chunks, blob = encode(L, ids, m.NL, m.NG)
        ql = synth.uniform(m.NL, 19 + variant)
        got = decode_and_gather(lim, rs, ci, info, chunks, blob, ql, m.NL, m.NG)
        assert np.array_equal(bits(got), bits(oracle.gather(ids, ql, m.NG)))
        if variant == 0:
            long_tiles = [t for t in range(info.shape[0] - 1) if info[t, 3] < 0]
            assert any(rs[info[t, 0] + 1] - rs[info[t, 0]] > lim[1] for t in long_tiles)
