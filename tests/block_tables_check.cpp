// Host-side checks of the tables a fused-block pass hands to block_pipe_kernel
// (built against the library by test_block_tables.py; no GPU needed).
//
// For random 5-qubit placements (and sliding windows) at 12..34 qubits:
//  * tile loads: simulating the loader's tensor boxes (box q covers the 128
//    amplitudes of bits 0..6 times the 2^g runs along positions g_lo.., at the
//    address bits q_off[q]) puts every address-order element e of the tile in
//    the shared-memory slot the producers read it from, (e & 127) | run_slot[e >> 7] << 7,
//    and fills every slot once;
//  * output staging: the index m*32 + (c ^ F(m)) built from the XOR tables equals
//    its definition, is a bijection, and the epilogue's staging writes (lanes =
//    32 consecutive rows, one column) and address-order reads (lanes = 32
//    consecutive elements) each hit 16 distinct 8-byte bank pairs;
//  * store walk: 16 Gray-code steps per thread over elements 256 k + et visit
//    every element once, with the address of each.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <set>
#include <vector>

#include "internal.h"

using namespace qs;

int main() {
  uint32_t rs = 12345u;
  auto rnd = [&]() {
    rs ^= rs << 13;
    rs ^= rs >> 17;
    rs ^= rs << 5;
    return rs;
  };
  long cases = 0, bad = 0;
  for (int n : {12, 13, 16, 20, 26, 30, 34}) {
    for (int t = 0; t < 600; ++t) {
      int bpos[5];
      std::vector<int> all(n);
      for (int i = 0; i < n; ++i) all[i] = i;
      for (int i = 0; i < 5; ++i) {
        const int k = i + (int)(rnd() % (uint32_t)(n - i));
        std::swap(all[i], all[k]);
        bpos[i] = all[i];
      }
      if (t % 3 == 0) {
        const int a = (int)(rnd() % (uint32_t)(n - 4));
        for (int i = 0; i < 5; ++i) bpos[i] = a + i;
      }
      std::sort(bpos, bpos + 5);
      BlockPass P;
      block_pass_desc(n, bpos, P);
      ++cases;
      long before = bad;
      if (!block_pass_runs_contiguous(P)) ++bad;
      auto addr = [&](int e) { return P.addr_lo[e & 63] | P.addr_hi[e >> 6]; };
      // ---- tile loads
      const int a = P.g_lo, g = P.g_len;
      if (a < 7 || g < 1 || a + g > n || P.n_copy != (1 << (5 - g))) {
        ++bad;
      } else {
        std::vector<long long> slot(4096, -1);
        for (int q = 0; q < P.n_copy; ++q) {
          const uint64_t A = P.q_off[q];
          if ((A & 127) || ((A >> a) & ((1ull << g) - 1))) ++bad;
          const uint64_t c1 = (A >> 7) & ((1ull << (a - 7)) - 1), c3 = A >> (a + g);
          for (int G = 0; G < (1 << g); ++G)
            for (int r = 0; r < 128; ++r) {
              const uint64_t ad = (uint64_t)r + 128ull * (c1 + (1ull << (a - 7)) * ((uint64_t)G + (1ull << g) * c3));
              const int so = ((q << g) | G) * 128 + r;
              if (slot[so] != -1) ++bad;
              slot[so] = (long long)ad;
            }
        }
        for (int e = 0; e < 4096; ++e)
          if (slot[(e & 127) | (P.run_slot[e >> 7] << 7)] != (long long)addr(e)) {
            ++bad;
            break;
          }
      }
      // ---- output staging
      auto F = [&](int m) {
        unsigned r = 0;
        for (int j = 0; j < 7; ++j)
          if ((m >> j) & 1) r ^= P.stage_f[j];
        return r & 31u;
      };
      auto mm = [&](int e) { return P.m_lo[e & 63] | P.m_hi[e >> 6]; };
      auto cc = [&](int e) { return P.c_lo[e & 63] | P.c_hi[e >> 6]; };
      unsigned sh[64];
      for (int v = 0; v < 64; ++v) sh[v] = (P.m_hi[v] << 5) ^ P.c_hi[v] ^ F(P.m_hi[v]);
      auto lo = [&](int v) { return (unsigned)((P.m_lo[v] << 5) ^ P.c_lo[v] ^ F(P.m_lo[v])); };
      auto idx = [&](int e) { return lo(e & 63) ^ sh[e >> 6]; };
      std::vector<int> seen(4096, 0);
      for (int e = 0; e < 4096; ++e) {
        if (idx(e) != mm(e) * 32u + (cc(e) ^ F(mm(e)))) ++bad;
        if (idx(e) < 4096) seen[idx(e)]++;
      }
      for (int i = 0; i < 4096; ++i)
        if (seen[i] != 1) {
          ++bad;
          break;
        }
      for (int e0 = 0; e0 < 4096; e0 += 32) {
        std::set<unsigned> banks;
        for (int l = 0; l < 32; ++l) banks.insert(idx(e0 + l) & 15);
        if (banks.size() != 16) ++bad;
      }
      for (int q = 0; q < 4; ++q)
        for (int c = 0; c < 32; ++c) {
          std::set<unsigned> banks;
          for (int l = 0; l < 32; ++l) banks.insert(((32 * q + l) * 32 + (c ^ F(32 * q + l))) & 15);
          if (banks.size() != 16) ++bad;
        }
      // ---- store walk
      std::vector<int> cov(4096, 0);
      for (int et = 0; et < 256; ++et) {
        uint64_t ad = (uint64_t)(et & 63) | P.addr_hi[et >> 6];
        unsigned ix = lo(et & 63) ^ sh[et >> 6];
        for (int k = 0; k < 16; ++k) {
          if (k) {
            const int b = (k & 1) ? 0 : (k & 2) ? 1 : (k & 4) ? 2 : 3;
            ad ^= P.addr_hi[4 << b];
            ix ^= sh[4 << b];
          }
          const int e = 256 * (k ^ (k >> 1)) + et;
          if (ad != addr(e) || ix != idx(e)) ++bad;
          cov[e]++;
        }
      }
      for (int e = 0; e < 4096; ++e)
        if (cov[e] != 1) {
          ++bad;
          break;
        }
      if (bad != before)
        std::printf("failed: n=%d block %d %d %d %d %d\n", n, bpos[0], bpos[1], bpos[2], bpos[3], bpos[4]);
    }
  }
  std::printf("cases %ld failures %ld\n", cases, bad);
  return bad != 0;
}
