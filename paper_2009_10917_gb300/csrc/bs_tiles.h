// bs_tiles.h -- the pipelined gather's per-tile re-encoding of the map
// (host code, plain C++: the library builds it in bs_map_create, and the host
// tests compile it on its own to check the encoding against the oracle).
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

namespace bs {

constexpr int kAgChunks = 512;    // chunks of two q_L values per tile
constexpr int kAgEntries = 1024;  // CSR entries per tile
constexpr int kAgRows = 768;      // rows per tile
constexpr int kAgBlob16 =
    ((kAgEntries + 7) / 8 * 8 + (kAgRows + 1 + 7) / 8 * 8 + (kAgRows + 7) / 8 * 8) * 2 / 16;

// One tile: first row, first chunk, first blob word (16 bytes), and
// (entries << 16 | rows), or -1 for rows summed straight from the CSR; the
// layout of the kernel's int4.
struct AgInfo {
  int32_t row, chunk, blob, meta;
};

// The pipelined gather's tiles (bs_gather.cuh): consecutive rows while the
// tile holds at most kAgEntries CSR entries, kAgRows rows and kAgChunks
// distinct chunks of two q_L values (local nodes 2c, 2c + 1); per tile the sorted chunk ids, then a blob
// of uint16 entry offsets (slot * 2 + the value's half of its chunk) and
// uint16 row starts relative to the tile's first entry, then the tile's rows
// (uint16, relative to its first row) in the order the kernel sums them, each
// part padded to 8 values.  A row that alone exceeds a tile gets a tile of its
// own marked -1.  With N_L odd the chunk of the last local node would run
// past q_L, so the row holding that node (one row at most) gets a tile of
// its own marked -1 as well and no chunk covers it.
struct AgTiles {
  std::vector<AgInfo> info;
  std::vector<int32_t> chunks;
  std::vector<uint16_t> blob;
};

inline AgTiles build_async_tiles(const std::vector<int32_t> &rs, const std::vector<int32_t> &col,
                                 int64_t NL, int64_t NG) {
  AgTiles T;
  std::vector<int32_t> mark((size_t)((NL + 1) / 2), -1);
  std::vector<int32_t> ch;
  int32_t tile = 0;
  // N_L odd: the row holding local node N_L - 1, summed straight from the CSR
  int64_t direct_row = -1;
  if (NL % 2 == 1)
    for (int64_t g = 0; g < NG && direct_row < 0; ++g)
      if (rs[(size_t)g] < rs[(size_t)g + 1] && col[(size_t)rs[(size_t)g + 1] - 1] == NL - 1)
        direct_row = g;
  auto row_chunks_new = [&](int64_t r) {  // chunks of row r not yet in the tile
    int fresh = 0;
    for (int32_t k = rs[(size_t)r]; k < rs[(size_t)r + 1]; ++k) {
      const int32_t c = col[(size_t)k] >> 1;
      if (mark[(size_t)c] == tile) continue;
      bool dup = false;
      for (int32_t q = rs[(size_t)r]; q < k && !dup; ++q) dup = (col[(size_t)q] >> 1) == c;
      fresh += !dup;
    }
    return fresh;
  };
  for (int64_t g = 0; g < NG;) {
    int64_t r = g;
    ch.clear();
    while (r < NG && r != direct_row && r - g < kAgRows &&
           rs[(size_t)r + 1] - rs[(size_t)g] <= kAgEntries &&
           (int)ch.size() + row_chunks_new(r) <= kAgChunks) {
      for (int32_t k = rs[(size_t)r]; k < rs[(size_t)r + 1]; ++k) {
        const int32_t c = col[(size_t)k] >> 1;
        if (mark[(size_t)c] != tile) {
          mark[(size_t)c] = tile;
          ch.push_back(c);
        }
      }
      ++r;
    }
    AgInfo in;
    in.row = (int32_t)g;
    in.chunk = (int32_t)T.chunks.size();
    in.blob = (int32_t)(T.blob.size() / 8);
    if (r == g) {  // one row too long for a tile, or the row of the odd last node
      in.meta = -1;
      r = g + 1;
    } else {
      std::sort(ch.begin(), ch.end());
      const int32_t k0 = rs[(size_t)g], nk = rs[(size_t)r] - k0;
      in.meta = (nk << 16) | (int32_t)(r - g);
      T.chunks.insert(T.chunks.end(), ch.begin(), ch.end());
      for (int32_t k = k0; k < k0 + nk; ++k) {
        const int32_t c = col[(size_t)k] >> 1;
        const int32_t slot = (int32_t)(std::lower_bound(ch.begin(), ch.end(), c) - ch.begin());
        T.blob.push_back((uint16_t)(slot * 2 + (col[(size_t)k] & 1)));
      }
      while (T.blob.size() % 8) T.blob.push_back(0);
      for (int64_t q = g; q <= r; ++q) T.blob.push_back((uint16_t)(rs[(size_t)q] - k0));
      while (T.blob.size() % 8) T.blob.push_back(0);
      // the summing order: rows by length, longest first (stable)
      std::vector<int32_t> ord((size_t)(r - g));
      for (size_t q = 0; q < ord.size(); ++q) ord[q] = (int32_t)q;
      auto len = [&](int32_t q) { return rs[(size_t)g + q + 1] - rs[(size_t)g + q]; };
      std::stable_sort(ord.begin(), ord.end(),
                       [&](int32_t a, int32_t b) { return len(a) > len(b); });
      for (int32_t q : ord) T.blob.push_back((uint16_t)q);
      while (T.blob.size() % 8) T.blob.push_back(0);
    }
    T.info.push_back(in);
    ++tile;
    g = r;
  }
  AgInfo last;
  last.row = (int32_t)NG;
  last.chunk = (int32_t)T.chunks.size();
  last.blob = (int32_t)(T.blob.size() / 8);
  last.meta = 0;
  T.info.push_back(last);
  return T;
}

}  // namespace bs
