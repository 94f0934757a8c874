// clut.cpp — object-mask compression (Sec. 3.2.2 compression LUT, Sec. 3.2.3
// requirement LUTs and Alg. 3).
//
// Table selection: the importance of a mask is SA(N) * O_m(N) / R^3 (the
// per-node term of Eq. 2), summed over the slots that use it (in slot
// order); the K most important distinct masks are kept (ties: mask value
// ascending), with an all-ones mask always present (it is a superset of
// every mask, so each slot has a conservative entry); the table is sorted
// by popcount ascending (then importance descending, value ascending) so
// that the lowest set bit of a candidate list is the tightest entry.
// Encoding: requirement LUT (i, p) = entries whose chunk i contains every
// bit of pattern p; a mask's entry = LSB of the AND over its chunks.
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace sc {
namespace {

struct Cand {
  const uint32_t* m;
  double imp;
  int pop;
};

int cmp_value(const uint32_t* a, const uint32_t* b, int W) {
  for (int w = W - 1; w >= 0; --w) {
    if (a[w] != b[w]) return a[w] < b[w] ? -1 : 1;
  }
  return 0;
}

inline uint64_t hash_mask(const uint32_t* m, int W) {
  uint64_t h = 1469598103934665603ULL;
  for (int w = 0; w < W; ++w) {
    h ^= m[w];
    h *= 1099511628211ULL;
    h ^= h >> 29;
  }
  return h;
}

inline int popcnt(const uint32_t* m, int W) {
  int c = 0;
  for (int w = 0; w < W; ++w) c += __builtin_popcount(m[w]);
  return c;
}

inline double slot_area(const float* b) {
  double dx = (double)b[3] - (double)b[0];
  double dy = (double)b[4] - (double)b[1];
  double dz = (double)b[5] - (double)b[2];
  return 2.0 * ((dx * dy + dy * dz) + dz * dx);
}

// Open-addressing set of distinct masks for one hash shard.
struct Shard {
  std::vector<int64_t> table;  // slot index of the first occurrence, -1 empty
  std::vector<Cand> cands;
  std::vector<int64_t> first;
};

}  // namespace

void build_compression(Bvh& b, int K, int bits, int threads) {
  double t0 = now_ms();
  const int W = b.W, R = b.R, R3 = R * R * R;
  const int64_t ns = b.nn * 2;
  b.compress = 1;
  b.bits = bits;
  // 1. distinct masks and summed importance, sharded by hash; each shard
  //    scans the slots in order, so sums follow slot order.
  const int S = std::max(1, std::min(64, threads));
  std::vector<uint64_t> hs((size_t)ns);
  parallel_for(ns, threads, 8192, [&](int64_t s) { hs[s] = hash_mask(&b.masks[(size_t)s * W], W); });
  std::vector<Shard> shards(S);
  parallel_for(S, threads, 1, [&](int64_t si) {
    Shard& sh = shards[si];
    size_t cap = 1024;
    while (cap < (size_t)(2 * ns / S + 16)) cap <<= 1;
    sh.table.assign(cap, -1);
    for (int64_t s = 0; s < ns; ++s) {
      uint64_t h = hs[s];
      if ((int64_t)(h % (uint64_t)S) != si) continue;
      const uint32_t* m = &b.masks[(size_t)s * W];
      double imp = (slot_area(&b.box[6 * s]) * (double)popcnt(m, W)) / (double)R3;
      size_t pos = (size_t)(h >> 8) & (cap - 1);
      for (;;) {
        int64_t e = sh.table[pos];
        if (e < 0) {
          sh.table[pos] = (int64_t)sh.cands.size();
          sh.cands.push_back(Cand{m, imp, popcnt(m, W)});
          break;
        }
        if (std::memcmp(sh.cands[e].m, m, sizeof(uint32_t) * W) == 0) {
          sh.cands[e].imp += imp;
          break;
        }
        pos = (pos + 1) & (cap - 1);
      }
    }
  });
  std::vector<Cand> all;
  for (auto& sh : shards) all.insert(all.end(), sh.cands.begin(), sh.cands.end());
  auto by_imp = [&](const Cand& a, const Cand& c) {
    if (a.imp != c.imp) return a.imp > c.imp;
    return cmp_value(a.m, c.m, W) < 0;
  };
  int64_t take = std::min<int64_t>((int64_t)all.size(), K);
  std::partial_sort(all.begin(), all.begin() + take, all.end(), by_imp);
  // 2. the all-ones entry
  std::vector<uint32_t> ones((size_t)W, 0u);
  for (int i = 0; i < R3; ++i) ones[i >> 5] |= 1u << (i & 31);
  bool has_ones = false;
  for (int64_t i = 0; i < take; ++i)
    if (std::memcmp(all[i].m, ones.data(), 4 * W) == 0) has_ones = true;
  std::vector<Cand> table(all.begin(), all.begin() + take);
  if (!has_ones) {
    double ones_imp = 0.0;
    for (size_t i = take; i < all.size(); ++i)
      if (std::memcmp(all[i].m, ones.data(), 4 * W) == 0) ones_imp = all[i].imp;
    if (take == K) table.pop_back();
    table.push_back(Cand{ones.data(), ones_imp, R3});
  }
  // 3. popcount order
  std::sort(table.begin(), table.end(), [&](const Cand& a, const Cand& c) {
    if (a.pop != c.pop) return a.pop < c.pop;
    return by_imp(a, c);
  });
  b.K = (int)table.size();
  b.clut.assign((size_t)b.K * W, 0u);
  for (int j = 0; j < b.K; ++j) std::memcpy(&b.clut[(size_t)j * W], table[j].m, 4 * W);
  encode_slots(b, threads, nullptr);
  b.ms_compress = now_ms() - t0;
}

// Alg. 3 for the slots of the nodes marked in node_dirty (every slot when
// NULL) against the LUT in b.clut: the requirement LUTs of Sec. 3.2.3, then
// per slot the first entry every chunk of its mask allows.
void encode_slots(Bvh& b, int threads, const std::vector<uint8_t>* node_dirty) {
  const int W = b.W, R = b.R, R3 = R * R * R, bits = b.bits;
  const int64_t ns = b.nn * 2;
  // 4. requirement LUTs: req[i][p] = 256-bit list of entries
  const int nchunk = (R3 + bits - 1) / bits, np = 1 << bits;
  auto chunk_of = [&](const uint32_t* m, int i) -> unsigned {
    unsigned v = 0;
    for (int j = 0; j < bits; ++j) {
      int bit = i * bits + j;
      if (bit < R3 && ((m[bit >> 5] >> (bit & 31)) & 1u)) v |= 1u << j;
    }
    return v;
  };
  std::vector<uint32_t> req((size_t)nchunk * np * 8, 0u);
  parallel_for(nchunk, threads, 1, [&](int64_t i) {
    for (int j = 0; j < b.K; ++j) {
      unsigned cj = chunk_of(&b.clut[(size_t)j * W], (int)i);
      for (int p = 0; p < np; ++p)
        if ((cj & (unsigned)p) == (unsigned)p)
          req[((size_t)i * np + p) * 8 + (j >> 5)] |= 1u << (j & 31);
    }
  });
  // 5. Alg. 3 for every (marked) slot
  if (!node_dirty) b.cidx.assign((size_t)ns, 0);
  const bool bytewise = (bits == 8);
  parallel_for(ns, threads, 4096, [&](int64_t s) {
    if (node_dirty && !(*node_dirty)[s >> 1]) return;
    const uint32_t* m = &b.masks[(size_t)s * W];
    const uint8_t* bytes = reinterpret_cast<const uint8_t*>(m);
    uint32_t list[8];
    for (int w = 0; w < 8; ++w) list[w] = 0xFFFFFFFFu;
    for (int i = 0; i < nchunk; ++i) {
      unsigned p = bytewise ? bytes[i] : chunk_of(m, i);
      const uint32_t* r = &req[((size_t)i * np + p) * 8];
      for (int w = 0; w < 8; ++w) list[w] &= r[w];
    }
    int idx = -1;
    for (int w = 0; w < 8 && idx < 0; ++w)
      if (list[w]) idx = 32 * w + __builtin_ctz(list[w]);
    if (idx < 0) fail(SC_ERR_STATE, "compression: no conservative LUT entry");
    b.cidx[s] = (uint8_t)idx;
  });
}

}  // namespace sc
