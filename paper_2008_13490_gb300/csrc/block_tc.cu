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
// Per tile (one CTA of 128 threads, persistent over tiles):
//   global -> registers (coalesced order) -> split -> shared memory (K-major,
//   no-swizzle core-matrix layout) -> tcgen05.mma x (K/8 or K/16) x 3 -> commit
//   to an mbarrier -> tcgen05.ld (thread = row) -> shared staging -> global.
// Every wait on the mbarrier is bounded; on timeout the kernel records
// QS_ETIMEOUT in a status word, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "internal.h"

namespace qs {

// ---------------------------------------------------------------- modes

enum : int { BM_TF32 = 0, BM_BF16 = 1 };

constexpr int kBlkThreads = 128;
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

__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float* v) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
      "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
      "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]),
        "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]),
        "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]),
        "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]),
        "=r"(r[62]), "=r"(r[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// ---------------------------------------------------------------- kernel

template <int MODE>
__global__ void __launch_bounds__(kBlkThreads)
    block_gemm_kernel(float2* __restrict__ psi, const BlockPass* __restrict__ P,
                      const unsigned char* __restrict__ bmat, uint64_t ntiles, int* __restrict__ status) {
  using O = BOps<MODE>;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* A_hi = smem;
  unsigned char* A_lo = smem + O::kA;
  unsigned char* B_hi = smem + 2 * O::kA;
  unsigned char* B_lo = B_hi + O::kB;
  float2* stage = reinterpret_cast<float2*>(smem);   // 32 KiB staging, reuses A after the MMAs
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base_slot;
  __shared__ uint64_t s_addr_lo[64], s_addr_hi[64];
  __shared__ uint8_t s_m_lo[64], s_m_hi[64], s_c_lo[64], s_c_hi[64], s_nt[48];
  __shared__ int s_nnt;
  const int tid = threadIdx.x, warp = tid >> 5;

  for (int i = tid; i < 64; i += kBlkThreads) {
    s_addr_lo[i] = P->addr_lo[i];
    s_addr_hi[i] = P->addr_hi[i];
    s_m_lo[i] = P->m_lo[i];
    s_m_hi[i] = P->m_hi[i];
    s_c_lo[i] = P->c_lo[i];
    s_c_hi[i] = P->c_hi[i];
  }
  if (tid < 48) s_nt[tid] = P->nt_pos[tid];
  if (tid == 0) s_nnt = P->n_nt;
  // B (hi, lo) in the core-matrix layout, prepared on the host
  {
    const uint4* src = reinterpret_cast<const uint4*>(bmat);
    uint4* dst = reinterpret_cast<uint4*>(B_hi);
    for (int i = tid; i < 2 * O::kB / 16; i += kBlkThreads) dst[i] = src[i];
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
                     smem_u32(&tmem_base_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem_d = tmem_base_slot;
  const uint32_t idesc = make_idesc<MODE>();
  uint32_t phase = 0;
  bool failed = false;

  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    uint64_t base = 0;
    for (int j = 0; j < s_nnt; ++j) base |= ((tile >> j) & 1ull) << s_nt[j];
    // ---- load (consecutive threads = consecutive low physical bits; all 32
    // loads in flight before the first use) and split
    float2 ld[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int e = i * kBlkThreads + tid;
      ld[i] = __ldcs(psi + (base | s_addr_lo[e & 63] | s_addr_hi[e >> 6]));
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int e = i * kBlkThreads + tid;
      const int lo = e & 63, hi = e >> 6;
      const int m = s_m_lo[lo] | s_m_hi[hi];
      const int c = s_c_lo[lo] | s_c_hi[hi];
      const float2 a = ld[i];
      if (MODE == BM_TF32) {
        const uint32_t hx = tf32_rna(a.x), hy = tf32_rna(a.y);
        const uint32_t lx = tf32_rna(a.x - __uint_as_float(hx)), ly = tf32_rna(a.y - __uint_as_float(hy));
        const uint32_t off = core_off<MODE>(m, 2 * c);
        *reinterpret_cast<uint2*>(A_hi + off) = make_uint2(hx, hy);
        *reinterpret_cast<uint2*>(A_lo + off) = make_uint2(lx, ly);
      } else {
        const __nv_bfloat16 hx = __float2bfloat16_rn(a.x), hy = __float2bfloat16_rn(a.y);
        const __nv_bfloat16 lx = __float2bfloat16_rn(a.x - __bfloat162float(hx));
        const __nv_bfloat16 ly = __float2bfloat16_rn(a.y - __bfloat162float(hy));
        const uint32_t off = core_off<MODE>(m, 2 * c);
        __nv_bfloat162 h2, l2;
        h2.x = hx;
        h2.y = hy;
        l2.x = lx;
        l2.y = ly;
        *reinterpret_cast<__nv_bfloat162*>(A_hi + off) = h2;
        *reinterpret_cast<__nv_bfloat162*>(A_lo + off) = l2;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // ---- MMAs into three FP32 accumulators: D1a / D1b = A_hi B_hi over the low /
    // high half of K (columns 0..63 / 128..191) and D2 = A_lo B_lo + A_hi B_lo +
    // A_lo B_hi (columns 64..127, smallest first).  The large product is summed
    // in short chains, so accumulator rounding adds few steps to it.
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hi = smem_u32(A_hi), a_lo = smem_u32(A_lo);
      const uint32_t b_hi = smem_u32(B_hi), b_lo = smem_u32(B_lo);
      constexpr int ksteps = 64 / O::kKStep;
      constexpr uint32_t kstep_bytes = 256;   // two K-adjacent core matrices
      for (int ks = 0; ks < ksteps; ++ks) {
        const uint32_t d = ks < ksteps / 2 ? tmem_d : tmem_d + 128;
        const uint64_t da = make_desc(a_hi + ks * kstep_bytes, 128, O::kSBO_A);
        const uint64_t db = make_desc(b_hi + ks * kstep_bytes, 128, O::kSBO_A);   // same K = 64
        mma<MODE>(d, da, db, idesc, (ks % (ksteps / 2)) ? 1u : 0u);
      }
      const uint32_t pa[3] = {a_lo, a_hi, a_lo};
      const uint32_t pb[3] = {b_lo, b_lo, b_hi};
      for (int p = 0; p < 3; ++p)
        for (int ks = 0; ks < ksteps; ++ks) {
          const uint64_t da = make_desc(pa[p] + ks * kstep_bytes, 128, O::kSBO_A);
          const uint64_t db = make_desc(pb[p] + ks * kstep_bytes, 128, O::kSBO_A);
          mma<MODE>(tmem_d + 64, da, db, idesc, (p > 0 || ks > 0) ? 1u : 0u);
        }
      mma_commit(smem_u32(&mbar));
    }
    // ---- wait (bounded) for the MMAs
    bool done = false;
    for (uint32_t it = 0; it < kWaitLimit; ++it)
      if (mbar_try_wait(smem_u32(&mbar), phase)) {
        done = true;
        break;
      }
    phase ^= 1u;
    if (__syncthreads_or(!done)) {
      failed = true;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- D = D1 + D2, row per thread -> staging in shared memory
    const int m = tid;
    const uint32_t lane_base = tmem_d + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float d1[32], d2[32];
      tmem_ld32(lane_base + 32 * h, d1);
      tmem_ld32(lane_base + 64 + 32 * h, d2);
#pragma unroll
      for (int j = 0; j < 32; ++j) d2[j] += d1[j];    // corrections + low-K half
      tmem_ld32(lane_base + 128 + 32 * h, d1);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int r = 16 * h + j;
        stage[m * 32 + (r ^ (m & 31))] = make_float2(d1[2 * j] + d2[2 * j], d1[2 * j + 1] + d2[2 * j + 1]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // ---- store in the load order
#pragma unroll 4
    for (int i = 0; i < 32; ++i) {
      const int e = i * kBlkThreads + tid;
      const int lo = e & 63, hi = e >> 6;
      const int mm = s_m_lo[lo] | s_m_hi[hi];
      const int c = s_c_lo[lo] | s_c_hi[hi];
      __stcs(psi + (base | s_addr_lo[lo] | s_addr_hi[hi]), stage[mm * 32 + (c ^ (mm & 31))]);
    }
    __syncthreads();
  }
  if (failed && tid == 0) atomicExch(status, (int)QS_ETIMEOUT);
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem_d) : "memory");
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

qs_status launch_block_pass(State* st, const void* pass_dev, const void* b_dev, int mode,
                            int* status_dev) {
  const uint64_t ntiles = 1ull << (st->n - 12);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // Each CTA holds 256 tensor-memory columns (three 64-column accumulators), so
  // at most 2 CTAs may share an SM (512 columns): the dynamic shared memory is
  // sized to enforce that residency limit, and the grid is 2 CTAs per SM.
  constexpr size_t kTwoPerSm = 96 * 1024;
  uint64_t grid = (uint64_t)sms * 2;
  if (grid > ntiles) grid = ntiles;
  if (mode == BM_TF32) {
    size_t smem = 2 * BOps<BM_TF32>::kA + 2 * BOps<BM_TF32>::kB;
    if (smem < kTwoPerSm) smem = kTwoPerSm;
    QS_CUDA(cudaFuncSetAttribute(block_gemm_kernel<BM_TF32>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    block_gemm_kernel<BM_TF32><<<(unsigned)grid, kBlkThreads, smem, st->stream>>>(
        (float2*)st->data, (const BlockPass*)pass_dev, (const unsigned char*)b_dev, ntiles, status_dev);
  } else {
    size_t smem = 2 * BOps<BM_BF16>::kA + 2 * BOps<BM_BF16>::kB;
    if (smem < kTwoPerSm) smem = kTwoPerSm;   // also covers the 32 KiB staging
    QS_CUDA(cudaFuncSetAttribute(block_gemm_kernel<BM_BF16>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    block_gemm_kernel<BM_BF16><<<(unsigned)grid, kBlkThreads, smem, st->stream>>>(
        (float2*)st->data, (const BlockPass*)pass_dev, (const unsigned char*)b_dev, ntiles, status_dev);
  }
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

}  // namespace qs
