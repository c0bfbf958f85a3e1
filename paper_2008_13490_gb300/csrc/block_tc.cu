// Fused 5-qubit blocks applied as complex GEMMs on the tcgen05 tensor cores.
//
// A block is the product of consecutive gates acting on at most 5 qubits, a
// dense 32x32 unitary U (the circuit is a product of small matrices, section
// "Quantum circuits"; here runs of them are multiplied on the host).  A tile of
// the state = 12 qubits: the block's 5 (columns c) and 7 others (rows m), 128
// rows x 32 complex amplitudes.  The update y_m = U x_m of every row is the real
// GEMM  D[128 x 64] = A[128 x 64] . B^T, A = (Re x_c, Im x_c) interleaved,
// B[n][k] = the real 64x64 form of U:
//   B[2r][2c] = Re U_rc,  B[2r][2c+1] = -Im U_rc,  B[2r+1][2c] = Im U_rc,  B[2r+1][2c+1] = Re U_rc.
// Operands are split into hi + lo parts (TF32 or BF16) and the product is
// A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation in tensor memory.
//
// Per tile (persistent CTAs, one per SM, the three stages overlapped over
// consecutive tiles by warp specialisation, see the kernel):
//   global -> registers (coalesced order) -> split -> shared memory (K-major,
//   no-swizzle core-matrix layout) -> tcgen05.mma x (K/8 or K/16) x 4 -> commit
//   to an mbarrier -> tcgen05.ld (thread = row) -> shared staging -> global.
// Every mbarrier wait is bounded; on timeout the kernel records QS_ETIMEOUT in
// a status word, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "internal.h"

namespace qs {

// ---------------------------------------------------------------- modes

enum : int { BM_TF32 = 0, BM_BF16 = 1 };

constexpr int kBlkRows = 128;
constexpr uint32_t kWaitLimit = 1u << 20;   // mbarrier polls before giving up (well under a second)

// byte sizes of one operand buffer
template <int MODE>
struct BOps;
template <>
struct BOps<BM_TF32> {
  static constexpr int kElem = 4;
  static constexpr int kKStep = 8;                 // K per tcgen05.mma (tf32)
  static constexpr int kSBO_A = 2048;              // 8-row group stride of A (K = 64 tf32)
  static constexpr int kA = kBlkRows * 64 * 4;     // 32 KiB
  static constexpr int kB = 64 * 64 * 4;           // 16 KiB
};
template <>
struct BOps<BM_BF16> {
  static constexpr int kElem = 2;
  static constexpr int kKStep = 16;
  static constexpr int kSBO_A = 1024;
  static constexpr int kA = kBlkRows * 64 * 2;     // 16 KiB
  static constexpr int kB = 64 * 64 * 2;           // 8 KiB
};

// byte offset of element (row, k) in a K-major no-swizzle core-matrix layout:
// core matrices of 8 rows x 16 bytes, K-adjacent cores 128 B apart (LBO),
// 8-row groups SBO apart
template <int MODE>
__host__ __device__ __forceinline__ uint32_t core_off(int row, int k) {
  constexpr int per = 16 / BOps<MODE>::kElem;   // elements per core row
  constexpr int sbo = 64 / per * 128;            // K = 64
  return (uint32_t)((row >> 3) * sbo + (k / per) * 128 + (row & 7) * 16 + (k % per) * BOps<MODE>::kElem);
}

// ---------------------------------------------------------------- PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version (tcgen05)
  // base offset 0, lbo mode 0, layout type 0 = no swizzle
  return d;
}

template <int MODE>
__device__ __forceinline__ uint32_t make_idesc() {
  // D = F32, A/B = TF32 (2) or BF16 (1), both K-major, N = 64, M = 128
  const uint32_t fmt = MODE == BM_TF32 ? 2u : 1u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
}

template <int MODE>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accumulate) {
  if (MODE == BM_TF32) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  }
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// ---------------------------------------------------------------- kernel
//
// One persistent CTA per SM, four roles that overlap consecutive tiles:
//   warp 9, one thread  loader: bulk-copies tile i into raw stage i % kStages of
//                       a shared-memory ring.  The 7 lowest physical bits are
//                       always tile bits (each is a block bit or one of the 7
//                       lowest others), so a tile is 32 contiguous runs of 128
//                       amplitudes (1 KiB each).
//   warps 0-3           producers: thread = row m; split row m of tile i into
//                       hi/lo parts, write it to operand buffer i % kABuf and
//                       free the raw stage for the loader
//   warp 8, one thread  MMA issuer: products of tile i into accumulator set i % 2
//   warps 4-7           epilogue: thread = row m = tensor-memory lane (warp w
//                       reads lanes 32*(w%4)..); add the partial sums, stage the
//                       rows in shared memory, store them to global memory in
//                       address order
// Hand-offs are mbarriers (full/empty per raw stage, per operand buffer and per
// accumulator set).  Every wait is bounded; a role that gives up sets a shared
// failure flag (which ends the other roles' waits early), the loader and the
// MMA issuer drain what they issued, and the kernel records QS_ETIMEOUT, frees
// its tensor memory and returns.

constexpr int kPipeThreads = 320;
constexpr int kTileBytes = 4096 * 8;          // one raw tile (complex64)
constexpr int kRun = 1024;                    // bytes of one contiguous run
constexpr int kEpiBarrier = 1;                // named barriers of the 128 epilogue threads:
constexpr int kEpiSync = 2;                   // reduction (kEpiBarrier) and plain sync

// Raw stages in flight and operand buffers (hi + lo each), within 224 KiB of
// shared memory together with B (hi + lo) and the 32 KiB output staging.
template <int MODE>
struct Pipe;
template <>
struct Pipe<BM_TF32> {
  static constexpr int kStages = 3;
  static constexpr int kABuf = 1;
};
template <>
struct Pipe<BM_BF16> {
  static constexpr int kStages = 4;
  static constexpr int kABuf = 1;
};
template <int MODE>
constexpr size_t pipe_smem_bytes() {
  return (size_t)(Pipe<MODE>::kStages + 1) * kTileBytes + (size_t)Pipe<MODE>::kABuf * 2 * BOps<MODE>::kA +
         2 * (size_t)BOps<MODE>::kB;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(b))
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(b))
      : "memory");
}
// bounded wait; gives up after kWaitLimit polls or, if fail is given, once
// another role has failed
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, const int* fail) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    if (mbar_try_wait(smem_u32(b), parity)) return true;
    if (fail && (it & 255u) == 255u && *reinterpret_cast<const volatile int*>(fail)) return false;
  }
  return false;
}
// OR of a predicate over the threads of a named barrier (all of them arrive)
__device__ __forceinline__ bool bar_or(int id, int nthreads, bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 q, %1, 0;\nbar.red.or.pred p, %2, %3, q;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}

template <int MODE>
__global__ void __launch_bounds__(kPipeThreads, 1)
    block_pipe_kernel(float2* __restrict__ psi, const BlockPass* __restrict__ P,
                      const unsigned char* __restrict__ bmat, uint64_t ntiles, int* __restrict__ status) {
  using O = BOps<MODE>;
  constexpr int kABuf = Pipe<MODE>::kABuf;
  constexpr int kStages = Pipe<MODE>::kStages;
  extern __shared__ __align__(1024) unsigned char smem[];
  // raw stage s at smem + s kTileBytes; operand buffer b: A_hi at abase + 2b kA,
  // A_lo at abase + (2b + 1) kA; then B_hi, B_lo
  unsigned char* abase = smem + kStages * kTileBytes;
  unsigned char* B_hi = abase + kABuf * 2 * O::kA;
  unsigned char* B_lo = B_hi + O::kB;
  float2* stage = reinterpret_cast<float2*>(B_lo + O::kB);   // 128 x 32 output amplitudes
  __shared__ __align__(8) uint64_t rfull[kStages], rempty[kStages], afull[2], aempty[2], tfull[2],
      tempty[2], drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  __shared__ uint64_t s_addr_lo[64], s_addr_hi[64];
  __shared__ uint8_t s_m_lo[64], s_m_hi[64], s_c_lo[64], s_c_hi[64], s_nt[48];
  __shared__ uint16_t s_em[128], s_ec[32];   // address-order index = s_em[m] | s_ec[c]
  // staging index m*32 + (c ^ (m & 31)) of the element with address-order
  // index e = the XOR of a term of its low 6 bits and s_sh[e >> 6] (the row and
  // column bits of the two halves are disjoint, so | and + become ^)
  __shared__ uint16_t s_sh[64];
  __shared__ int s_nnt;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int i = tid; i < 64; i += kPipeThreads) {
    s_addr_lo[i] = P->addr_lo[i];
    s_addr_hi[i] = P->addr_hi[i];
    s_m_lo[i] = P->m_lo[i];
    s_m_hi[i] = P->m_hi[i];
    s_c_lo[i] = P->c_lo[i];
    s_c_hi[i] = P->c_hi[i];
  }
  if (tid < 48) s_nt[tid] = P->nt_pos[tid];
  if (tid == 0) {
    s_nnt = P->n_nt;
    s_fail = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&rfull[s], 1);
      mbar_init(&rempty[s], 128);   // producers
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&afull[b], 128);
      mbar_init(&aempty[b], 1);
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 128);
    }
    mbar_init(&drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    const uint4* src = reinterpret_cast<const uint4*>(bmat);
    uint4* dst = reinterpret_cast<uint4*>(B_hi);
    for (int i = tid; i < 2 * O::kB / 16; i += kPipeThreads) dst[i] = src[i];
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  for (int e = tid; e < 4096; e += kPipeThreads) {
    const int m = s_m_lo[e & 63] | s_m_hi[e >> 6], c = s_c_lo[e & 63] | s_c_hi[e >> 6];
    if (c == 0) s_em[m] = (uint16_t)e;
    if (m == 0) s_ec[c] = (uint16_t)e;
  }
  if (tid < 64) s_sh[tid] = (uint16_t)((s_m_hi[tid] << 5) ^ s_c_hi[tid] ^ (s_m_hi[tid] & 31));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  auto tile_base = [&](uint64_t i) {
    const uint64_t tile = blockIdx.x + i * gridDim.x;
    uint64_t base = 0;
    for (int j = 0; j < s_nnt; ++j) base |= ((tile >> j) & 1ull) << s_nt[j];
    return base;
  };

  if (warp == 9) {
    // ---------------- loader (one warp; lane j copies run j of the tile)
    uint64_t issued = 0;
    const uint64_t run_off = s_addr_hi[2 * lane];
    for (uint64_t i = 0; i < my_tiles; ++i) {
      const int s = (int)(i % kStages);
      const uint32_t ph = (uint32_t)((i / kStages) & 1);
      const bool ok = mbar_wait(&rempty[s], ph ^ 1u, &s_fail);
      if (__any_sync(0xffffffffu, !ok)) {
        if (lane == 0) atomicExch(&s_fail, 1);
        break;
      }
      const uint64_t base = tile_base(i);
      if (lane == 0) mbar_arrive_tx(&rfull[s], kTileBytes);   // before any of the copies
      __syncwarp();
      bulk_load(smem + s * kTileBytes + lane * kRun, psi + (base | run_off), kRun, &rfull[s]);
      issued = i + 1;
    }
    // no copy may still be writing shared memory when the CTA exits
    if (lane == 0)
      for (uint64_t t = issued > (uint64_t)kStages ? issued - kStages : 0; t < issued; ++t)
        if (!mbar_wait(&rfull[t % kStages], (uint32_t)((t / kStages) & 1), nullptr))
          atomicExch(&s_fail, 1);
  } else if (warp < 4) {
    // ---------------- producers: thread = row m; groups of G columns fill one
    // 16-byte core-matrix row each, groups in a lane-rotated order (the 32 lanes
    // of a write then cover the 8 rows of a core matrix 4 times: no conflicts
    // beyond the 4 wavefronts of 512 bytes)
    constexpr int G = MODE == BM_TF32 ? 2 : 4;
    constexpr int NG = 32 / G;
    const int m = tid;
    const int rot = m & (NG - 1);
    // The address-order index of (m, c) is s_em[m] | s_ec[c], and s_ec deposits
    // the bits of c, so it is linear over XOR: the index of column
    // (jj ^ rot) G + u is e0 ^ ecg[jj] ^ ecu[u] with per-thread registers.
    uint32_t ecg[NG], ecu[G];
#pragma unroll
    for (int jj = 0; jj < NG; ++jj) ecg[jj] = s_ec[jj * G];
#pragma unroll
    for (int u = 0; u < G; ++u) ecu[u] = s_ec[u];
    const uint32_t e0 = s_em[m] ^ s_ec[rot * G];
    // byte offset of group g in row m: core_off(m, 2 G g) = row_off + 128 g
    const uint32_t row_off = core_off<MODE>(m, 0);
    for (uint64_t i = 0; i < my_tiles; ++i) {
      const int s = (int)(i % kStages);
      const uint32_t ph = (uint32_t)((i / kStages) & 1);
      const int b = (int)(i % kABuf);
      const uint32_t pa = (uint32_t)((i / kABuf) & 1);
      if (!mbar_wait(&rfull[s], ph, &s_fail) || !mbar_wait(&aempty[b], pa ^ 1u, &s_fail)) {
        atomicExch(&s_fail, 1);
        break;
      }
      const float2* raw = reinterpret_cast<const float2*>(smem + s * kTileBytes);
      unsigned char* Ah = abase + b * 2 * O::kA + row_off;
      unsigned char* Al = Ah + O::kA;
#pragma unroll
      for (int jj = 0; jj < NG; ++jj) {
        float v[2 * G];   // Re, Im of columns gG .. gG+G-1, g = jj ^ rot
#pragma unroll
        for (int u = 0; u < G; ++u) {
          const float2 a = raw[e0 ^ ecg[jj] ^ ecu[u]];
          v[2 * u] = a.x;
          v[2 * u + 1] = a.y;
        }
        uint32_t hw[4], lw[4];
        if (MODE == BM_TF32) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            hw[q] = tf32_rna(v[q]);
            lw[q] = tf32_rna(v[q] - __uint_as_float(hw[q]));
          }
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
            const float2 hf = __bfloat1622float2(h2);
            const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[2 * q] - hf.x, v[2 * q + 1] - hf.y);
            hw[q] = *reinterpret_cast<const uint32_t*>(&h2);
            lw[q] = *reinterpret_cast<const uint32_t*>(&l2);
          }
        }
        const uint32_t off = (uint32_t)(jj ^ rot) << 7;   // 16-byte aligned
        *reinterpret_cast<uint4*>(Ah + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(Al + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&afull[b]);
      mbar_arrive(&rempty[s]);   // raw stage s may be refilled
    }
  } else if (warp == 8) {
    // ---------------- MMA issuer (one thread)
    if (lane == 0) {
      const uint32_t idesc = make_idesc<MODE>();
      const uint32_t b_hi = smem_u32(B_hi), b_lo = smem_u32(B_lo);
      constexpr int ksteps = 64 / O::kKStep;
      constexpr uint32_t kstep_bytes = 256;   // two K-adjacent core matrices
      for (uint64_t i = 0; i < my_tiles; ++i) {
        const int b = (int)(i % kABuf);
        const uint32_t pa = (uint32_t)((i / kABuf) & 1);
        const int tb = (int)(i & 1);
        const uint32_t pt = (uint32_t)((i >> 1) & 1);
        if (!mbar_wait(&afull[b], pa, &s_fail) || !mbar_wait(&tempty[tb], pt ^ 1u, &s_fail)) {
          atomicExch(&s_fail, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a_hi = smem_u32(abase) + (uint32_t)(b * 2 * O::kA), a_lo = a_hi + O::kA;
        // three FP32 accumulators: D1a / D1b = A_hi B_hi over the low / high half
        // of K (columns +0 / +128), D2 = A_lo B_lo + A_hi B_lo + A_lo B_hi (+64,
        // smallest first); the large product is summed in short chains
        const uint32_t d = tmem + 256u * (uint32_t)tb;
        for (int ks = 0; ks < ksteps; ++ks) {
          const uint32_t dd = ks < ksteps / 2 ? d : d + 128;
          mma<MODE>(dd, make_desc(a_hi + ks * kstep_bytes, 128, O::kSBO_A),
                    make_desc(b_hi + ks * kstep_bytes, 128, O::kSBO_A), idesc,
                    (ks % (ksteps / 2)) ? 1u : 0u);
        }
        const uint32_t pa3[3] = {a_lo, a_hi, a_lo};
        const uint32_t pb3[3] = {b_lo, b_lo, b_hi};
#pragma unroll
        for (int p = 0; p < 3; ++p)
          for (int ks = 0; ks < ksteps; ++ks)
            mma<MODE>(d + 64, make_desc(pa3[p] + ks * kstep_bytes, 128, O::kSBO_A),
                      make_desc(pb3[p] + ks * kstep_bytes, 128, O::kSBO_A), idesc,
                      (p > 0 || ks > 0) ? 1u : 0u);
        mma_commit(smem_u32(&aempty[b]));   // operand buffer b may be refilled
        mma_commit(smem_u32(&tfull[tb]));   // accumulator set tb is ready
      }
      // every product issued above has finished before the tensor memory is freed
      mma_commit(smem_u32(&drain));
      if (!mbar_wait(&drain, 0, nullptr)) atomicExch(&s_fail, 1);
    }
  } else {
    // ---------------- epilogue (warps 4..7)
    const int m = (warp & 3) * 32 + lane;   // row of the tile = tensor-memory lane
    const int et = tid - 128;               // 0..127, store order
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const int m_lo = s_m_lo[et & 63], c_lo = s_c_lo[et & 63];
    const uint32_t sh_lo = (uint32_t)((m_lo << 5) ^ c_lo ^ (m_lo & 31));
    // run k = 0 of this thread, and the change of address / staging index when
    // bit b of k flips (element index bit 7 + b = address-order high half bit 1 + b)
    const uint64_t addr0 = s_addr_lo[et & 63] | s_addr_hi[et >> 6];
    const uint32_t idx0 = sh_lo ^ s_sh[et >> 6];
    uint64_t dA[5];
    uint32_t dS[5];
#pragma unroll
    for (int bit = 0; bit < 5; ++bit) {
      dA[bit] = s_addr_hi[2 << bit];
      dS[bit] = s_sh[2 << bit];
    }
    for (uint64_t i = 0; i < my_tiles; ++i) {
      const int tb = (int)(i & 1);
      const uint32_t pt = (uint32_t)((i >> 1) & 1);
      const bool ok = mbar_wait(&tfull[tb], pt, &s_fail);
      // collective: all 128 epilogue threads stop together (and none of them is
      // still reading the staging of the previous tile past this point)
      if (bar_or(kEpiBarrier, 128, !ok)) {
        atomicExch(&s_fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t d = tmem + lane_base + 256u * (uint32_t)tb;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float d1[32], d2[32];
        tmem_ld32(d + 32 * h, d1);
        tmem_ld32(d + 64 + 32 * h, d2);
#pragma unroll
        for (int j = 0; j < 32; ++j) d2[j] += d1[j];    // corrections + low-K half
        tmem_ld32(d + 128 + 32 * h, d1);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = 16 * h + j;
          stage[m * 32 + (c ^ (m & 31))] = make_float2(d1[2 * j] + d2[2 * j], d1[2 * j + 1] + d2[2 * j + 1]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&tempty[tb]);   // accumulator set tb may be overwritten
      asm volatile("bar.sync %0, %1;" ::"r"(kEpiSync), "r"(128) : "memory");
      // element k * 128 + et for the runs k in Gray-code order: the address and
      // the staging index are XOR-linear in the bits of k, so each step flips one
      uint64_t addr = tile_base(i) | addr0;
      uint32_t idx = idx0;
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        if (t) {
          const int bit = (t & 1) ? 0 : (t & 2) ? 1 : (t & 4) ? 2 : (t & 8) ? 3 : 4;   // lowest set bit
          addr ^= dA[bit];
          idx ^= dS[bit];
        }
        __stcs(psi + addr, stage[idx]);
      }
    }
  }
  __syncthreads();
  if (tid == 0 && s_fail) atomicExch(status, (int)QS_ETIMEOUT);
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ---------------------------------------------------------------- host side

namespace {

// rounds to the tf32 grid (10 explicit mantissa bits), nearest, ties away from zero
float tf32_round_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;
  u += 0x1000u;
  u &= 0xffffe000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

uint16_t bf16_round_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;   // round to nearest even
  return (uint16_t)(u >> 16);
}

float bf16_to_float(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

}  // namespace

// Fills the B operand (hi then lo) of a block in the kernel's shared-memory layout.
void block_b_operand(const cd* U, int mode, std::vector<unsigned char>& out) {
  double W[64][64];   // W[n][k] (B is N x K, K-major)
  for (int r = 0; r < 32; ++r)
    for (int c = 0; c < 32; ++c) {
      const double re = U[r * 32 + c].real(), im = U[r * 32 + c].imag();
      W[2 * r][2 * c] = re;
      W[2 * r][2 * c + 1] = -im;
      W[2 * r + 1][2 * c] = im;
      W[2 * r + 1][2 * c + 1] = re;
    }
  if (mode == BM_TF32) {
    const int kB = BOps<BM_TF32>::kB;
    out.assign(2 * kB, 0);
    for (int n = 0; n < 64; ++n)
      for (int k = 0; k < 64; ++k) {
        const float x = (float)W[n][k];
        const float h = tf32_round_host(x);
        const float l = tf32_round_host((float)(W[n][k] - (double)h));
        const uint32_t off = core_off<BM_TF32>(n, k);
        std::memcpy(out.data() + off, &h, 4);
        std::memcpy(out.data() + kB + off, &l, 4);
      }
  } else {
    const int kB = BOps<BM_BF16>::kB;
    out.assign(2 * kB, 0);
    for (int n = 0; n < 64; ++n)
      for (int k = 0; k < 64; ++k) {
        const uint16_t h = bf16_round_host((float)W[n][k]);
        const uint16_t l = bf16_round_host((float)(W[n][k] - (double)bf16_to_float(h)));
        const uint32_t off = core_off<BM_BF16>(n, k);
        std::memcpy(out.data() + off, &h, 2);
        std::memcpy(out.data() + kB + off, &l, 2);
      }
  }
}

size_t block_b_bytes(int mode) { return mode == BM_TF32 ? 2 * BOps<BM_TF32>::kB : 2 * BOps<BM_BF16>::kB; }

// Tile bookkeeping: block bits (5 physical positions, local block bit i = bit i
// of the column index) and 7 row positions (the lowest other positions).
void block_pass_desc(int n, const int* bpos, BlockPass& P) {
  std::memset(&P, 0, sizeof(P));
  bool in_block[64] = {};
  for (int i = 0; i < 5; ++i) in_block[bpos[i]] = true;
  int rows[7], nr = 0;
  for (int p = 0; p < n && nr < 7; ++p)
    if (!in_block[p]) rows[nr++] = p;
  bool in_tile[64] = {};
  for (int i = 0; i < 5; ++i) in_tile[bpos[i]] = true;
  for (int i = 0; i < 7; ++i) in_tile[rows[i]] = true;
  // address order: the 12 tile positions ascending
  int order[12], no = 0;
  for (int p = 0; p < n; ++p)
    if (in_tile[p]) order[no++] = p;
  int nt = 0;
  for (int p = 0; p < n; ++p)
    if (!in_tile[p]) P.nt_pos[nt++] = (uint8_t)p;
  P.n_nt = nt;
  auto role = [&](int p, int* is_col, int* idx) {
    for (int i = 0; i < 5; ++i)
      if (bpos[i] == p) {
        *is_col = 1;
        *idx = i;
        return;
      }
    for (int i = 0; i < 7; ++i)
      if (rows[i] == p) {
        *is_col = 0;
        *idx = i;
        return;
      }
  };
  for (int v = 0; v < 64; ++v) {
    for (int half = 0; half < 2; ++half) {
      uint64_t addr = 0;
      int m = 0, c = 0;
      for (int j = 0; j < 6; ++j) {
        if (!((v >> j) & 1)) continue;
        const int p = order[half * 6 + j];
        addr |= 1ull << p;
        int is_col = 0, idx = 0;
        role(p, &is_col, &idx);
        if (is_col) c |= 1 << idx;
        else m |= 1 << idx;
      }
      if (half == 0) {
        P.addr_lo[v] = addr;
        P.m_lo[v] = (uint8_t)m;
        P.c_lo[v] = (uint8_t)c;
      } else {
        P.addr_hi[v] = addr;
        P.m_hi[v] = (uint8_t)m;
        P.c_hi[v] = (uint8_t)c;
      }
    }
  }
}

size_t block_pass_bytes() { return sizeof(BlockPass); }

// The kernel's loader copies a tile as 32 runs of 128 amplitudes: the 7 lowest
// address-order bits must be the physical bits 0..6.
bool block_pass_runs_contiguous(const BlockPass& P) {
  for (int v = 0; v < 64; ++v)
    if (P.addr_lo[v] != (uint64_t)v) return false;
  return P.addr_hi[1] == 64;
}

qs_status launch_block_pass(State* st, const void* pass_dev, const void* b_dev, int mode,
                            int* status_dev) {
  const uint64_t ntiles = 1ull << (st->n - 12);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // Each CTA holds all 512 tensor-memory columns (two sets of three 64-column
  // accumulators, 256 columns apart), so exactly one CTA may run per SM: the
  // dynamic shared memory (raw ring, operand buffers, B: 208-224 KiB) is more
  // than half of the SM's, and the grid is one CTA per SM.
  static_assert(pipe_smem_bytes<BM_BF16>() > 120 * 1024, "one CTA per SM");
  static_assert(pipe_smem_bytes<BM_TF32>() <= 224 * 1024, "shared memory per CTA");
  uint64_t grid = (uint64_t)sms;
  if (grid > ntiles) grid = ntiles;
  if (mode == BM_TF32) {
    const size_t smem = pipe_smem_bytes<BM_TF32>();
    QS_CUDA(cudaFuncSetAttribute(block_pipe_kernel<BM_TF32>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    block_pipe_kernel<BM_TF32><<<(unsigned)grid, kPipeThreads, smem, st->stream>>>(
        (float2*)st->data, (const BlockPass*)pass_dev, (const unsigned char*)b_dev, ntiles, status_dev);
  } else {
    const size_t smem = pipe_smem_bytes<BM_BF16>();
    QS_CUDA(cudaFuncSetAttribute(block_pipe_kernel<BM_BF16>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    block_pipe_kernel<BM_BF16><<<(unsigned)grid, kPipeThreads, smem, st->stream>>>(
        (float2*)st->data, (const BlockPass*)pass_dev, (const unsigned char*)b_dev, ntiles, status_dev);
  }
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

}  // namespace qs
