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
// Operands are split into two TF32 or three BF16 parts and the product keeps
// the part products down to FP32 size, accumulated in FP32 in tensor memory.
//
// Per tile (persistent CTAs, one per SM, the stages overlapped over consecutive
// tiles by warp specialisation, see the kernel):
//   global -> bulk copy -> shared memory -> split -> shared memory (K-major,
//   no-swizzle core-matrix layout) -> tcgen05.mma -> commit to an mbarrier ->
//   tcgen05.ld (thread = row) -> shared staging -> global.
// Every mbarrier wait is bounded; on timeout the kernel records QS_ETIMEOUT in
// a status word, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "internal.h"

namespace qs {

// ---------------------------------------------------------------- modes

enum : int { BM_TF32 = 0, BM_BF16 = 1 };

constexpr int kBlkRows = 128;
constexpr uint32_t kWaitLimit = 1u << 20;   // mbarrier polls before giving up (well under a second)

// Operand formats.  An FP32 value x is split into parts x = x_0 + x_1 (+ x_2),
// each rounded to the MMA's input type: TF32 (11 significant bits) in two parts,
// BF16 (8 significant bits) in three, both keeping about 22-24 bits.  The
// product A.B keeps the part products down to about 2^-22 (TF32) or 2^-24 (BF16)
// relative size: A_0 B_0 and kNCorr correction products (a-part, b-part).
template <int MODE>
struct BOps;
template <>
struct BOps<BM_TF32> {
  static constexpr int kElem = 4;
  static constexpr int kKStep = 8;                 // K per tcgen05.mma (tf32)
  static constexpr int kSBO_A = 2048;              // 8-row group stride of A (K = 64 tf32)
  static constexpr int kA = kBlkRows * 64 * 4;     // one part of A: 32 KiB
  static constexpr int kB = 64 * 64 * 4;           // one part of B: 16 KiB
  static constexpr int kParts = 2;
  static constexpr int kNCorr = 3;                 // (1,1) (0,1) (1,0)
};
template <>
struct BOps<BM_BF16> {
  static constexpr int kElem = 2;
  static constexpr int kKStep = 16;
  static constexpr int kSBO_A = 1024;
  static constexpr int kA = kBlkRows * 64 * 2;     // 16 KiB
  static constexpr int kB = 64 * 64 * 2;           // 8 KiB
  static constexpr int kParts = 3;
  static constexpr int kNCorr = 5;                 // (2,0) (0,2) (1,1) (1,0) (0,1)
};
// correction product p (smallest first): parts of A and B
template <int MODE>
__host__ __device__ constexpr int corr_a(int p) {
  return MODE == BM_TF32 ? (p == 1 ? 0 : 1) : (p == 0 ? 2 : p == 1 ? 0 : p == 4 ? 0 : 1);
}
template <int MODE>
__host__ __device__ constexpr int corr_b(int p) {
  return MODE == BM_TF32 ? (p == 2 ? 0 : 1) : (p == 0 ? 0 : p == 1 ? 2 : p == 3 ? 0 : 1);
}

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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// tcgen05.ld without the wait: several loads share one tcgen05.wait::ld, after
// which reg_after_wait32 ties the registers to the wait (their uses cannot be
// scheduled before it)
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t* r) {
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
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void reg_after_wait32(uint32_t* r) {
  asm volatile(""
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                 "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]),
                 "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]),
                 "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]),
                 "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]),
                 "+r"(r[31]));
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// ---------------------------------------------------------------- kernel
//
// One persistent CTA per SM, four roles that overlap consecutive tiles:
//   warp 13             loader: tile i into raw stage i % kStages of a
//                       shared-memory ring, as 2^(5-g) tensor boxes.  The 7
//                       lowest physical bits are always tile bits (each is a
//                       block bit or one of the 7 lowest others), so a tile is
//                       32 contiguous runs of 128 amplitudes (1 KiB each); the
//                       other 5 tile positions hold a run of g consecutive
//                       ones, and one box copies the 2^g runs along it
//                       (1 KiB requests cost the copy engine far more per byte)
//   warps 0-3           producers: thread = row m = tensor-memory lane; split row
//                       m of tile i into its parts and store them into the A
//                       operand in tensor memory (tcgen05.st), one K half (16
//                       columns) at a time; note the row's squared norm and free
//                       the raw stage for the loader
//   warp 12, one thread MMA issuer: the products of each K half of tile i (A from
//                       tensor memory, B from shared memory) into accumulator set
//                       i % 2, as soon as that half is stored (the producer fills
//                       one half while the tensor cores read the other)
//   warps 4-11          epilogue: warps w and w + 4 share the tensor-memory lanes
//                       32*(w%4).. (thread = row m) and take 16 columns each; add
//                       the partial sums, rescale the row, stage the rows in
//                       shared memory, store them to global memory in address
//                       order
// With N = 64 an MMA that reads both operands from shared memory needs more
// bytes per cycle than shared memory delivers; A in tensor memory leaves only B
// (shared by all tiles) there.  Tensor-memory columns: accumulator set t at
// 256 t (D1a +0, D2 +64, D1b +128); A parts in the free columns 192..255 and
// 448..511.
// Hand-offs are mbarriers (full/empty per raw stage, per K half of the operand
// and per accumulator set).  Every wait is bounded; a role that gives up
// sets a shared failure flag (which ends the other roles' waits early), the
// loader and the MMA issuer drain what they issued, and the kernel records
// QS_ETIMEOUT, frees its tensor memory and returns.
//
// Norm correction: a unitary block maps every row x_m to a row U x_m of the same
// norm.  The tensor cores' FP32 accumulation loses a little magnitude on every
// pass (a bias that grows linearly with the number of blocks), so for blocks
// the host found unitary the epilogue rescales each output row to the squared
// norm of its input row, computed by the producer in FP32.

constexpr int kPipeThreads = 448;
constexpr int kEpiThreads = 256;
constexpr int kTileBytes = 4096 * 8;          // one raw tile (complex64)
constexpr int kRun = 1024;                    // bytes of one contiguous run
constexpr int kEpiBarrier = 1;                // named barriers of the 256 epilogue threads:
constexpr int kEpiSync = 2;                   // reduction (kEpiBarrier) and plain sync
constexpr int kEpiPair = 3;                   // 3..6: the two epilogue warps of one row range
constexpr int kNormSlots = 3;                 // row norms in flight (producer -> epilogue)
constexpr int kWarpMma = 12, kWarpLoad = 13;

// Raw stages in flight; shared memory = the raw ring, B and the 32 KiB output
// staging (TF32: 128 + 32 + 32 KiB; BF16: 128 + 24 + 32 KiB).
template <int MODE>
struct Pipe {
  static constexpr int kStages = 4;
};
// two output staging buffers (box-store passes alternate between them, so the
// tensor store of one tile may still be reading its buffer while the next tile is
// staged)
constexpr int kStageBufs = 2;
template <int MODE>
constexpr size_t pipe_smem_bytes() {
  return (size_t)(Pipe<MODE>::kStages + kStageBufs) * kTileBytes + (size_t)BOps<MODE>::kParts * BOps<MODE>::kB;
}
// tensor-memory column of part p of A (BF16: 32 columns per part, two bf16 per
// column; TF32: 64 columns per part)
template <int MODE>
__host__ __device__ constexpr uint32_t a_col(int p) {
  return MODE == BM_TF32 ? (p == 0 ? 192u : 448u) : (p == 0 ? 192u : p == 1 ? 224u : 448u);
}

template <int MODE>
__device__ __forceinline__ void mma_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  if (MODE == BM_TF32) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
        "r"(tmem_a), "l"(b), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
        "r"(tmem_a), "l"(b), "r"(idesc), "r"(accumulate));
  }
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// conditional swap of the complex entries j and j ^ 2^BIT of a 16-entry row
template <int BIT>
__device__ __forceinline__ void xswap16_bit(float2* x, bool sw) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << BIT)) continue;
    const int k = j | (1 << BIT);
    const float2 a = x[j], b = x[k];
    x[j] = sw ? b : a;
    x[k] = sw ? a : b;
  }
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
// one box of a rank-4 tensor map (coordinates innermost first) into shared memory
__device__ __forceinline__ void box_load4(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                          uint64_t* b) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
      "%4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(b))
      : "memory");
}
// one box of a rank-4 tensor map from shared memory to global memory (bulk group)
__device__ __forceinline__ void box_store4(const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                           const void* src) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
      : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the bulk groups of this thread but the newest one have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
// every bulk group of this thread has completed (its writes are done)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

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
__device__ __forceinline__ void bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 v) {
  return *reinterpret_cast<const uint32_t*>(&v);
}

// BOX: the pass writes its output back with tensor stores (BlockPass flag bit 1);
// a separate instantiation, so that each variant keeps its own register budget
template <int MODE, bool BOX>
__global__ void __launch_bounds__(kPipeThreads, 1)
    block_pipe_kernel(float2* __restrict__ psi, const BlockPass* __restrict__ P,
                      const unsigned char* __restrict__ bmat, uint64_t ntiles, int* __restrict__ status,
                      const __grid_constant__ CUtensorMap tmap) {
  using O = BOps<MODE>;
  constexpr int kStages = Pipe<MODE>::kStages;
  constexpr int kParts = O::kParts;
  extern __shared__ __align__(1024) unsigned char smem[];
  // raw stage s at smem + s kTileBytes; then B (part p at bbase + p kB) and the
  // output staging
  unsigned char* bbase = smem + kStages * kTileBytes;
  float2* stage = reinterpret_cast<float2*>(bbase + kParts * O::kB);   // 128 x 32 amplitudes
  // tables used only while the roles set up their registers, kept in the staging
  unsigned char* tab = reinterpret_cast<unsigned char*>(stage);
  uint64_t* t_addr_hi = reinterpret_cast<uint64_t*>(tab);              // 64 x 8 B
  uint8_t* t_m_lo = tab + 512;
  uint8_t* t_m_hi = tab + 576;
  uint8_t* t_c_lo = tab + 640;
  uint8_t* t_c_hi = tab + 704;
  uint16_t* t_em = reinterpret_cast<uint16_t*>(tab + 768);              // 128 x 2 B
  uint16_t* t_ec = reinterpret_cast<uint16_t*>(tab + 1024);             // 32 x 2 B
  uint16_t* t_sh = reinterpret_cast<uint16_t*>(tab + 1088);             // 64 x 2 B
  __shared__ __align__(8) uint64_t rfull[kStages], rempty[kStages], afull[2], aempty[2], tfull[2],
      tempty[2], drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  __shared__ uint8_t s_nt[48];
  __shared__ uint8_t s_slot[32];
  __shared__ uint8_t s_f[8];
  __shared__ int s_nnt;
  __shared__ uint64_t s_qoff[16];
  __shared__ int s_ncopy, s_glo, s_glen;
  __shared__ float s_norm[kNormSlots][128];   // producer -> epilogue: squared input row norms
  __shared__ float s_part[2][128];            // epilogue column halves: squared output norms
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool unitary = (P->flags & 1) != 0;
  // the output is staged in the loader's box layout and written back with tensor
  // stores (the host found the staging writes conflict-free in that layout)
  constexpr bool boxst = BOX;

  if (tid < 64) {
    t_addr_hi[tid] = P->addr_hi[tid];
    t_m_lo[tid] = P->m_lo[tid];
    t_m_hi[tid] = P->m_hi[tid];
    t_c_lo[tid] = P->c_lo[tid];
    t_c_hi[tid] = P->c_hi[tid];
  }
  if (tid < 48) s_nt[tid] = P->nt_pos[tid];
  if (tid < 32) s_slot[tid] = P->run_slot[tid];
  if (tid < 8) s_f[tid] = P->stage_f[tid];
  if (tid < 16) s_qoff[tid] = tid < P->n_copy ? P->q_off[tid] : 0ull;
  if (tid == 0) {
    s_nnt = P->n_nt;
    s_ncopy = P->n_copy;
    s_glo = P->g_lo;
    s_glen = P->g_len;
    s_fail = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&rfull[s], 1);
      mbar_init(&rempty[s], 128);   // producers
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&afull[b], 128);    // producers, per K half
      mbar_init(&aempty[b], 1);     // MMA commit, per K half
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiThreads);
    }
    mbar_init(&drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    const uint4* src = reinterpret_cast<const uint4*>(bmat);
    uint4* dst = reinterpret_cast<uint4*>(bbase);
    for (int i = tid; i < kParts * O::kB / 16; i += kPipeThreads) dst[i] = src[i];
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  for (int e = tid; e < 4096; e += kPipeThreads) {
    const int m = t_m_lo[e & 63] | t_m_hi[e >> 6], c = t_c_lo[e & 63] | t_c_hi[e >> 6];
    if (c == 0) t_em[m] = (uint16_t)e;
    if (m == 0) t_ec[c] = (uint16_t)e;
  }
  // staging index m*32 + (c ^ F(m)) of the element with address-order index
  // e = (term of its low 6 bits) ^ t_sh[e >> 6]: the row and column bits of the
  // two halves are disjoint, so | and + become ^ (F is XOR-linear)
  auto stage_F = [&](int m) {
    uint32_t r = 0;
#pragma unroll
    for (int j = 0; j < 7; ++j)
      if ((m >> j) & 1) r ^= s_f[j];
    return r;
  };
  if (tid < 64) t_sh[tid] = (uint16_t)((t_m_hi[tid] << 5) ^ t_c_hi[tid] ^ stage_F(t_m_hi[tid]));
  __syncthreads();

  // ---- per-role registers (from the tables; the staging is free after this)
  // producers: the address-order index of (m, c) is em[m] | ec[c], and ec
  // deposits the bits of c, so it is linear over XOR.  At step j of a K half the
  // thread reads column 16 h + (j ^ sigma): sigma(lane) feeds the lane bits that
  // the row bits leave free into the column bits sitting at address bits 0..3
  // (with the block's qubits in ascending order those are column bits
  // 0..ncb-1), so the 32 lanes of a read fall on 16 distinct 8-byte bank pairs;
  // a select network then puts column 16 h + j into slot j.
  uint32_t ecb[4], ec16 = 0, e00 = 0;   // ec[2^b], ec[16], the index of slot 0 of half 0
  int ncb = 0;
  // epilogue: element k * 256 + et of the store loop, k in Gray-code order: its
  // address and staging index at k = 0 and their change when bit b of k flips
  // (element bit 8 + b = bit 2 + b of the high half); F(m) of the row written
  // (box-store passes reuse idx0 / dS for the staging index in the raw-stage slot
  // layout of this row's first column and its change with column bits 0..3)
  uint64_t addr0 = 0, dA[4];
  uint32_t idx0 = 0, dS[4], fm = 0;
  // loader: lane q < n_copy loads box q: the address bits q_off of its runs
  // outside the box, and the box's position (bits 7..g_lo-1 and above g_lo+g_len
  // are the tensor coordinates 1 and 3)
  uint64_t q_off = 0;
  int n_copy = 0, g_lo = 7, g_len = 5;
  if (warp < 4) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
      if (t_c_lo[1 << a]) ++ncb;
    uint32_t sigma = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (r < ncb) sigma |= (uint32_t)((lane >> (4 - ncb + r)) & 1) << r;
#pragma unroll
    for (int b = 0; b < 4; ++b) ecb[b] = t_ec[1 << b];
    ec16 = t_ec[16];
    e00 = t_em[tid] ^ t_ec[sigma];
    // raw stages hold run j (address-order bits 7..11) in slot s_slot[j]: a bit
    // permutation, so it applies to the XOR steps as well
    auto slot = [&](uint32_t e) { return (e & 127u) | ((uint32_t)s_slot[e >> 7] << 7); };
#pragma unroll
    for (int b = 0; b < 4; ++b) ecb[b] = slot(ecb[b]);
    ec16 = slot(ec16);
    e00 = slot(e00);
  } else if (warp < 12) {
    if (boxst) {
      auto slot = [&](uint32_t e) { return (e & 127u) | ((uint32_t)s_slot[e >> 7] << 7); };
      const int half = (warp - 4) >> 2, mrow = (warp & 3) * 32 + lane;
      idx0 = slot((uint32_t)t_em[mrow] ^ (uint32_t)t_ec[16 * half]);
#pragma unroll
      for (int b = 0; b < 4; ++b) dS[b] = slot(t_ec[1 << b]);
    } else {
      const int et = tid - 128;   // 0..255
      const int m_lo = t_m_lo[et & 63], c_lo = t_c_lo[et & 63];
      addr0 = (uint64_t)(et & 63) | t_addr_hi[et >> 6];   // low 6 bits: physical bits 0..5
      idx0 = (uint32_t)((m_lo << 5) ^ c_lo ^ stage_F(m_lo)) ^ t_sh[et >> 6];
#pragma unroll
      for (int bit = 0; bit < 4; ++bit) {
        dA[bit] = t_addr_hi[4 << bit];
        dS[bit] = t_sh[4 << bit];
      }
      fm = stage_F((warp & 3) * 32 + lane) & 31u;
    }
  } else if (warp == kWarpLoad) {
    n_copy = P->n_copy;
    g_lo = P->g_lo;
    g_len = P->g_len;
    if (lane < n_copy) q_off = P->q_off[lane];
  }
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

  if (warp == kWarpLoad) {
    // ---------------- loader
    uint64_t issued = 0;
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
      if (lane < n_copy) {
        const uint64_t a = base | q_off;
        const int c1 = (int)((a >> 7) & ((1ull << (g_lo - 7)) - 1)), c3 = (int)(a >> (g_lo + g_len));
        box_load4(smem + s * kTileBytes + (lane << g_len) * kRun, &tmap, 0, c1, 0, c3, &rfull[s]);
      }
      issued = i + 1;
    }
    // no copy may still be writing shared memory when the CTA exits
    if (lane == 0)
      for (uint64_t t = issued > (uint64_t)kStages ? issued - kStages : 0; t < issued; ++t)
        if (!mbar_wait(&rfull[t % kStages], (uint32_t)((t / kStages) & 1), nullptr))
          atomicExch(&s_fail, 1);
  } else if (warp < 4) {
    // ---------------- producers: thread = row m = tensor-memory lane
    const int m = tid;
    const uint32_t tlane = (uint32_t)((warp & 3) * 32) << 16;
    for (uint64_t i = 0; i < my_tiles; ++i) {
      const int s = (int)(i % kStages);
      const uint32_t ph = (uint32_t)((i / kStages) & 1);
      const uint32_t pa = (uint32_t)(i & 1);
      // warp-uniform outcomes: the tensor-memory stores below are warp-collective
      const bool okr = mbar_wait(&rfull[s], ph, &s_fail);
      if (__any_sync(0xffffffffu, !okr)) {
        atomicExch(&s_fail, 1);
        break;
      }
      const float2* raw = reinterpret_cast<const float2*>(smem + s * kTileBytes);
      // the whole row first (32 independent loads; slot j of half h at x[16 h + j],
      // slots visited in Gray-code order: one XOR per step)
      float2 x[32];
      {
        uint32_t e = e00;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          if (t) e ^= ecb[(t & 1) ? 0 : (t & 2) ? 1 : (t & 4) ? 2 : 3];
          const int j = t ^ (t >> 1);
          x[j] = raw[e];
          x[16 + j] = raw[e ^ ec16];
        }
      }
      mbar_arrive(&rempty[s]);   // the row is in registers: raw stage s may be refilled
      float nrm[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        nrm[(2 * j) & 3] = fmaf(x[j].x, x[j].x, nrm[(2 * j) & 3]);
        nrm[(2 * j + 1) & 3] = fmaf(x[j].y, x[j].y, nrm[(2 * j + 1) & 3]);
      }
      // keep the norm here: sunk to its store it would keep a copy of the row alive
      asm volatile("" : "+f"(nrm[0]), "+f"(nrm[1]), "+f"(nrm[2]), "+f"(nrm[3]));
      // slot j <- column 16 h + j
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (ncb > 0) xswap16_bit<0>(x + 16 * h, ((lane >> (4 - ncb)) & 1) != 0);
        if (ncb > 1) xswap16_bit<1>(x + 16 * h, ((lane >> (5 - ncb)) & 1) != 0);
        if (ncb > 2) xswap16_bit<2>(x + 16 * h, ((lane >> (6 - ncb)) & 1) != 0);
        if (ncb > 3) xswap16_bit<3>(x + 16 * h, ((lane >> 3) & 1) != 0);
      }
      bool ok = true;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float2* xh = x + 16 * h;
        // the tensor cores have finished reading this K half of the previous tile
        const bool oka = mbar_wait(&aempty[h], pa ^ 1u, &s_fail);
        if (__any_sync(0xffffffffu, !oka)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // each part is rounded from the running residual, which stays exact in
        // FP32, and stored before the next part is formed
        uint32_t w[16];
        if constexpr (MODE == BM_TF32) {
          // K index 2c (Re) and 2c + 1 (Im) at columns a_col(p) + 32 h + ..
#pragma unroll
          for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                float2& v = xh[8 * q + j];
                w[2 * j] = tf32_rna(v.x);
                w[2 * j + 1] = tf32_rna(v.y);
                v.x -= __uint_as_float(w[2 * j]);
                v.y -= __uint_as_float(w[2 * j + 1]);
              }
              tmem_st16(tmem + tlane + a_col<MODE>(p) + 32u * h + 16u * q, w);
            }
        } else {
          // three bf16 parts; column a_col(p) + 16 h + j holds (Re, Im) of column 16 h + j
#pragma unroll
          for (int p = 0; p < 3; ++p) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const __nv_bfloat162 b2 = __floats2bfloat162_rn(xh[j].x, xh[j].y);
              w[j] = bf16x2_bits(b2);
              if (p < 2) {
                const float2 bf = __bfloat1622float2(b2);
                xh[j].x -= bf.x;
                xh[j].y -= bf.y;
              }
            }
            tmem_st16(tmem + tlane + a_col<MODE>(p) + 16u * h, w);
          }
        }
        tmem_wait_st();
        if (h == 1) s_norm[i % kNormSlots][m] = (nrm[0] + nrm[1]) + (nrm[2] + nrm[3]);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&afull[h]);
      }
      if (!ok) {
        atomicExch(&s_fail, 1);
        break;
      }
    }
  } else if (warp == kWarpMma) {
    // ---------------- MMA issuer (one thread)
    if (lane == 0) {
      const uint32_t idesc = make_idesc<MODE>();
      const uint32_t b0 = smem_u32(bbase);
      constexpr int ksteps = 64 / O::kKStep;
      constexpr int khalf = ksteps / 2;
      constexpr uint32_t kstep_bytes = 256;   // two K-adjacent core matrices
      for (uint64_t i = 0; i < my_tiles; ++i) {
        const uint32_t pa = (uint32_t)(i & 1);
        const int tb = (int)(i & 1);
        const uint32_t pt = (uint32_t)((i >> 1) & 1);
        if (!mbar_wait(&tempty[tb], pt ^ 1u, &s_fail)) {
          atomicExch(&s_fail, 1);
          break;
        }
        // three FP32 accumulators: D1a / D1b = A_0 B_0 over the low / high half
        // of K (columns +0 / +128) and D2 = the correction products (+64), each
        // half's smallest first; the large product is summed in short chains
        const uint32_t d = tmem + 256u * (uint32_t)tb;
        bool ok = true;
        for (int h = 0; h < 2; ++h) {
          if (!mbar_wait(&afull[h], pa, &s_fail)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          // A: 8 tensor-memory columns per K step (8 tf32 or 16 bf16)
          for (int ks = h * khalf; ks < (h + 1) * khalf; ++ks)
            mma_ta<MODE>(d + 128u * (uint32_t)h, tmem + a_col<MODE>(0) + 8u * ks,
                         make_desc(b0 + ks * kstep_bytes, 128, O::kSBO_A), idesc, ks > h * khalf ? 1u : 0u);
#pragma unroll
          for (int p = 0; p < O::kNCorr; ++p) {
            const uint32_t ap = tmem + a_col<MODE>(corr_a<MODE>(p));
            const uint32_t bp = b0 + (uint32_t)(corr_b<MODE>(p) * O::kB);
            for (int ks = h * khalf; ks < (h + 1) * khalf; ++ks)
              mma_ta<MODE>(d + 64, ap + 8u * ks, make_desc(bp + ks * kstep_bytes, 128, O::kSBO_A), idesc,
                           (h > 0 || p > 0 || ks > 0) ? 1u : 0u);
          }
          mma_commit(smem_u32(&aempty[h]));   // this K half of the operand buffer may be refilled
        }
        if (!ok) {
          atomicExch(&s_fail, 1);
          break;
        }
        mma_commit(smem_u32(&tfull[tb]));   // accumulator set tb is ready
      }
      // every product issued above has finished before the tensor memory is freed
      mma_commit(smem_u32(&drain));
      if (!mbar_wait(&drain, 0, nullptr)) atomicExch(&s_fail, 1);
    }
  } else {
    // ---------------- epilogue (warps 4..11)
    const int half = (warp - 4) >> 2;            // complex columns 16 half .. 16 half + 15
    const int m = (warp & 3) * 32 + lane;       // row of the tile = tensor-memory lane
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const bool leader = tid == 128;   // issues and waits for the tensor stores
    for (uint64_t i = 0; i < my_tiles; ++i) {
      const int tb = (int)(i & 1);
      const uint32_t pt = (uint32_t)((i >> 1) & 1);
      // box store: the store of tile i - 2 has read staging buffer i % 2 (the
      // barrier below publishes that to the other epilogue threads)
      if (boxst && leader) bulk_wait_read_1();
      const bool okw = mbar_wait(&tfull[tb], pt, &s_fail);
      // collective: all epilogue threads stop together (and none of them is
      // still reading the staging or s_part of the previous tile past this point)
      if (bar_or(kEpiBarrier, kEpiThreads, !okw)) {
        atomicExch(&s_fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const float nx = s_norm[i % kNormSlots][m];
      const uint32_t d = tmem + lane_base + 256u * (uint32_t)tb + 32u * (uint32_t)half;
      // y = (D2 + D1a) + D1b over this warp's 32 float columns
      float y[32];
      {
        uint32_t a[32], b[32];
        tmem_ld32_nowait(d + 64, a);
        tmem_ld32_nowait(d, b);
        tmem_wait_ld();
        reg_after_wait32(a);
        reg_after_wait32(b);
#pragma unroll
        for (int j = 0; j < 32; ++j) y[j] = __uint_as_float(a[j]) + __uint_as_float(b[j]);
        tmem_ld32_nowait(d + 128, b);
        tmem_wait_ld();
        reg_after_wait32(b);
#pragma unroll
        for (int j = 0; j < 32; ++j) y[j] += __uint_as_float(b[j]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&tempty[tb]);   // accumulator set tb may be overwritten
      // y <- y (1 + delta), 1 + delta = sqrt(nx / ny).  delta is formed as
      // (nx - ny) / (ny + sqrt(nx ny)) (nx - ny is exact when they are close) and
      // added with one fma: a factor rounded to FP32 near 1 (spacing 2^-23 above
      // 1, and sqrt(1 + 2^-23) rounds back to 1) would drop the small
      // corrections systematically.  ny = the two halves' sums, in a fixed order.
      float delta = 0.f;
      if (unitary) {
        float sq[16];   // pairwise sum of this half's 32 squares
#pragma unroll
        for (int j = 0; j < 16; ++j) sq[j] = fmaf(y[2 * j], y[2 * j], y[2 * j + 1] * y[2 * j + 1]);
#pragma unroll
        for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
          for (int j = 0; j < w; ++j) sq[j] += sq[j + w];
        s_part[half][m] = sq[0];
        bar_sync(kEpiPair + (warp & 3), 64);   // the two warps of these rows
        const float ny = s_part[0][m] + s_part[1][m];
        if (ny > 0.f) delta = (nx - ny) / (ny + sqrtf(nx) * sqrtf(ny));
      }
      if (boxst) {
        // the loader's layout: column j of this half at bx0 ^ (XOR of bxd over the
        // set bits of j), visited in Gray-code order; lanes = rows, conflict-free
        float2* stg = stage + (i & 1) * 4096;
        uint32_t idx = idx0;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          if (t) idx ^= dS[(t & 1) ? 0 : (t & 2) ? 1 : (t & 4) ? 2 : 3];
          const int j = t ^ (t >> 1);
          stg[idx] = make_float2(fmaf(y[2 * j], delta, y[2 * j]), fmaf(y[2 * j + 1], delta, y[2 * j + 1]));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor store
        bar_sync(kEpiSync, kEpiThreads);
        if (leader) {
          const uint64_t base = tile_base(i);
          for (int q = 0; q < s_ncopy; ++q) {
            const uint64_t a = base | s_qoff[q];
            const int c1 = (int)((a >> 7) & ((1ull << (s_glo - 7)) - 1)), c3 = (int)(a >> (s_glo + s_glen));
            box_store4(&tmap, 0, c1, 0, c3, stg + (q << s_glen) * 128);
          }
          bulk_commit();
        }
        continue;
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = 16 * half + j;
        stage[m * 32 + (c ^ fm)] =
            make_float2(fmaf(y[2 * j], delta, y[2 * j]), fmaf(y[2 * j + 1], delta, y[2 * j + 1]));
      }
      bar_sync(kEpiSync, kEpiThreads);
      // (all staging reads first, then all stores)
      float2 v[16];
      {
        uint32_t idx = idx0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          if (k) idx ^= dS[(k & 1) ? 0 : (k & 2) ? 1 : (k & 4) ? 2 : 3];   // lowest set bit
          v[k] = stage[idx];
        }
      }
      uint64_t addr = tile_base(i) | addr0;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        if (k) addr ^= dA[(k & 1) ? 0 : (k & 2) ? 1 : (k & 4) ? 2 : 3];
        __stcs(psi + addr, v[k]);
      }
    }
    // no tensor store may still be reading shared memory (or writing) at exit
    if (boxst && leader) bulk_wait_all();
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

// Fills the B operand of a block (its parts one after another) in the kernel's
// shared-memory layout; the parts are split from the FP64 matrix.
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
    out.assign(3 * kB, 0);
    for (int n = 0; n < 64; ++n)
      for (int k = 0; k < 64; ++k) {
        double r = W[n][k];
        const uint32_t off = core_off<BM_BF16>(n, k);
        for (int p = 0; p < 3; ++p) {
          const uint16_t h = bf16_round_host((float)r);
          r -= (double)bf16_to_float(h);
          std::memcpy(out.data() + p * kB + off, &h, 2);
        }
      }
  }
}

size_t block_b_bytes(int mode) {
  return mode == BM_TF32 ? BOps<BM_TF32>::kParts * BOps<BM_TF32>::kB
                         : BOps<BM_BF16>::kParts * BOps<BM_BF16>::kB;
}

bool block_is_unitary(const cd* U) {
  // (U^dagger U)_ij = sum_k conj(U_ki) U_kj in real arithmetic; Hermitian, so j >= i
  double re[32][32], im[32][32];
  for (int k = 0; k < 32; ++k)
    for (int i = 0; i < 32; ++i) {
      re[k][i] = U[k * 32 + i].real();
      im[k][i] = U[k * 32 + i].imag();
    }
  for (int i = 0; i < 32; ++i)
    for (int j = i; j < 32; ++j) {
      double sr = 0, si = 0;
      for (int k = 0; k < 32; ++k) {
        sr += re[k][i] * re[k][j] + im[k][i] * im[k][j];
        si += re[k][i] * im[k][j] - im[k][i] * re[k][j];
      }
      if (i == j) sr -= 1.0;
      if (sr * sr + si * si > 1e-20) return false;
    }
  return true;
}

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
  // tensor-box loads: H = order[7..11]; the first longest run of consecutive
  // positions in H becomes the box's second dimension
  const int* H = order + 7;
  int g0 = 0, g = 1;
  for (int i = 0; i < 5;) {
    int k = i + 1;
    while (k < 5 && H[k] == H[k - 1] + 1) ++k;
    if (k - i > g) {
      g0 = i;
      g = k - i;
    }
    i = k;
  }
  P.g0 = g0;
  P.g_len = g;
  P.g_lo = H[g0];
  P.n_copy = 1 << (5 - g);
  for (int j = 0; j < 32; ++j) {
    const int lo = j & ((1 << g0) - 1), gv = (j >> g0) & ((1 << g) - 1), hi = j >> (g0 + g);
    P.run_slot[j] = (uint8_t)(gv | (lo << g) | (hi << (g + g0)));
  }
  for (int q = 0; q < P.n_copy; ++q) {
    const int j = (q & ((1 << g0) - 1)) | ((q >> g0) << (g0 + g));
    uint64_t off = 0;
    for (int b = 0; b < 5; ++b)
      if ((j >> b) & 1) off |= 1ull << H[b];
    P.q_off[q] = off;
  }
  // staging swizzle F: the bank pair of an 8-byte staging word is its index mod 16,
  // i.e. bits 0..3 of c ^ F(m).  Writes: a warp's lanes are row bits 0..4, so
  // {F(2^j) mod 16, j < 5} must span the 4 bits.  Reads: a warp's lanes are
  // physical bits 0..4; a column bit c_i there contributes 2^i (i < 4), a row bit
  // m_j contributes F(2^j) mod 16, and these must span the 4 bits.  F(2^j) = 2^j
  // (j < 5) is tried first, then a fixed pseudo-random sequence.
  auto rank4 = [](const uint32_t* v, int k) {
    uint32_t basis[4] = {0, 0, 0, 0};
    int r = 0;
    for (int i = 0; i < k; ++i) {
      uint32_t x = v[i] & 15u;
      for (int b = 3; b >= 0 && x; --b)
        if ((x >> b) & 1) {
          if (!basis[b]) {
            basis[b] = x;
            ++r;
            x = 0;
          } else {
            x ^= basis[b];
          }
        }
    }
    return r;
  };
  uint32_t F[7];
  uint32_t seed = 0x9e3779b9u;
  for (int trial = 0; trial < 4096; ++trial) {
    for (int j = 0; j < 7; ++j) {
      if (trial == 0) {
        F[j] = j < 5 ? (1u << j) & 15u : 0u;
      } else {
        seed ^= seed << 13;
        seed ^= seed >> 17;
        seed ^= seed << 5;
        F[j] = seed & 15u;
      }
    }
    uint32_t rd[5];
    for (int p = 0; p < 5; ++p) {
      int is_col = 0, idx = 0;
      role(p, &is_col, &idx);
      rd[p] = is_col ? (idx < 4 ? 1u << idx : 0u) : F[idx];
    }
    if (rank4(F, 5) == 4 && rank4(rd, 5) == 4) break;
    if (trial == 4095)
      for (int j = 0; j < 7; ++j) F[j] = j < 5 ? (1u << j) & 15u : 0u;   // (2-way conflicts)
  }
  for (int j = 0; j < 7; ++j) P.stage_f[j] = (uint8_t)F[j];
  P.stage_f[7] = 0;
  // box store: the epilogue writes row m, column c to the loader's slot of its
  // address-order index; a warp's lanes are row bits 0..4, so the writes meet 16
  // distinct 8-byte bank pairs when the slots of those row bits span bits 0..3
  uint32_t rowslot[5];
  for (int j = 0; j < 5; ++j) {
    int a = 0;
    while (order[a] != rows[j]) ++a;
    const uint32_t e = 1u << a;
    rowslot[j] = (e & 127u) | ((uint32_t)P.run_slot[e >> 7] << 7);
  }
  if (rank4(rowslot, 5) == 4) P.flags |= 2;
}

size_t block_pass_bytes() { return sizeof(BlockPass); }

// The kernel's loader copies a tile as 32 runs of 128 amplitudes: the 7 lowest
// address-order bits must be the physical bits 0..6.
bool block_pass_runs_contiguous(const BlockPass& P) {
  for (int v = 0; v < 64; ++v)
    if (P.addr_lo[v] != (uint64_t)v) return false;
  return P.addr_hi[1] == 64;
}

// The tensor map of a pass's tile loads: the state as [128 | 2^(g_lo-7) |
// 2^g_len | 2^(n-g_lo-g_len)] amplitudes (8 bytes each), box 128 x 1 x 2^g_len x 1.
static qs_status block_tensor_map(const State* st, const BlockPass& P, CUtensorMap* map) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      set_error("cuTensorMapEncodeTiled is not available");
      return QS_ECUDA;
    }
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  const int a = P.g_lo, g = P.g_len, n = st->n;
  if (a < 7 || g < 1 || a + g > n || P.n_copy != (1 << (5 - g))) {
    set_error("block pass: invalid tile box");
    return QS_EINVAL;
  }
  const cuuint64_t dims[4] = {128, 1ull << (a - 7), 1ull << g, 1ull << (n - a - g)};
  const cuuint64_t strides[3] = {1024, 8ull << a, 8ull << (a + g)};
  const cuuint32_t box[4] = {128, 1, 1u << g, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, st->data, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed for a block pass");
    return QS_ECUDA;
  }
  return QS_OK;
}

qs_status launch_block_pass(State* st, const BlockPass& host_pass, const void* pass_dev, const void* b_dev,
                            int mode, int* status_dev) {
  CUtensorMap map;
  const qs_status ms = block_tensor_map(st, host_pass, &map);
  if (ms != QS_OK) return ms;
  const uint64_t ntiles = 1ull << (st->n - 12);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // Each CTA holds all 512 tensor-memory columns (two sets of three 64-column
  // accumulators, 256 columns apart), so exactly one CTA may run per SM: the
  // dynamic shared memory (raw ring, B, staging: 184-192 KiB) is more than half
  // of the SM's, and the grid is one CTA per SM.
  static_assert(pipe_smem_bytes<BM_BF16>() > 120 * 1024, "one CTA per SM");
  static_assert(pipe_smem_bytes<BM_TF32>() <= 224 * 1024, "shared memory per CTA");
  static_assert(pipe_smem_bytes<BM_BF16>() <= 224 * 1024, "shared memory per CTA");
  // a CTA needs a whole SM: leave the SMs a server's persistent kernel may hold
  uint64_t grid = (uint64_t)std::max(1, sms - reserved_sms());
  if (grid > ntiles) grid = ntiles;
  const bool box = (host_pass.flags & 2) != 0;
  auto launch = [&](auto kern, size_t smem) -> qs_status {
    QS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)grid, kPipeThreads, smem, st->stream>>>((float2*)st->data, (const BlockPass*)pass_dev,
                                                             (const unsigned char*)b_dev, ntiles, status_dev, map);
    return QS_OK;
  };
  qs_status ls;
  if (mode == BM_TF32)
    ls = box ? launch(block_pipe_kernel<BM_TF32, true>, pipe_smem_bytes<BM_TF32>())
             : launch(block_pipe_kernel<BM_TF32, false>, pipe_smem_bytes<BM_TF32>());
  else
    ls = box ? launch(block_pipe_kernel<BM_BF16, true>, pipe_smem_bytes<BM_BF16>())
             : launch(block_pipe_kernel<BM_BF16, false>, pipe_smem_bytes<BM_BF16>());
  if (ls != QS_OK) return ls;
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

}  // namespace qs
