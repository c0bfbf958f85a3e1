// Internal declarations shared by the host runtime (.cpp) and the kernels (.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <string>
#include <vector>

#include "qsim.h"

namespace qs {

using cd = std::complex<double>;

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
qs_status cuda_status(cudaError_t e, const char* what);

#define QS_CUDA(call)                                           \
  do {                                                          \
    cudaError_t e__ = (call);                                   \
    if (e__ != cudaSuccess) return ::qs::cuda_status(e__, #call); \
  } while (0)

// ---------------------------------------------------------------- state
struct State {
  int n = 0;
  int prec = QS_C64;
  size_t amp_bytes = 8;         // bytes per amplitude
  void* data = nullptr;         // 2^n amplitudes
  size_t data_bytes = 0;
  bool owns_data = true;        // false: a caller's buffer (sv_wrap), not freed here
  void* scratch = nullptr;      // reduction partials + small device tables
  size_t scratch_bytes = 0;
  cudaStream_t stream = nullptr;
  qs_allocator alloc{};
  bool has_alloc = false;
  int device = 0;
  // device op buffer reused between calls (grown on demand)
  void* opbuf = nullptr;
  size_t opbuf_bytes = 0;
  // pinned host staging buffer for op uploads
  void* hostbuf = nullptr;
  size_t hostbuf_bytes = 0;
  cudaEvent_t upload_done = nullptr;
  // device staging buffer of probabilities bound for host memory (sv_probs_host)
  void* stage = nullptr;
  size_t stage_bytes = 0;
};

void* dev_alloc(State* st, size_t bytes);
void dev_free(State* st, void* p, size_t bytes);
qs_status ensure_opbuf(State* st, size_t bytes);

// Per-state scratch (device): reduction partials, counters, small tables.
constexpr int kReduceBlocks = 1024;               // partial sums written by reduction kernels
constexpr size_t kScratchPartials = 0;            // kReduceBlocks doubles
constexpr size_t kScratchClamps = 8192;           // one 64-bit counter
constexpr size_t kScratchResult = 8448;           // 16 doubles
constexpr size_t kScratchBits = 8704;             // 64 bytes of bit positions
constexpr size_t kScratchMarg = 16384;            // marginal accumulators (doubles)
constexpr int kScratchMargLog2 = 16;              // largest marginal kept in scratch
constexpr size_t kScratchBytes = kScratchMarg + (sizeof(double) << kScratchMargLog2);
// staging buffer of sv_probs_host (allocated at its first call, kept by the state)
constexpr size_t kStageBytes = 64ull << 20;

// ---------------------------------------------------------------- gates
// Host-side gate matrices, written from the thesis's definitions (rotations,
// U gates, Tab. (elementarygateset), CNOT, CZ, CP, SWAP).  dim = 2 or 4.
bool gate_matrix(const qs_gate& g, cd* m, int* dim);
// d/dparam[k] of the gate matrix (parameterised kinds only).
bool gate_dmatrix(const qs_gate& g, int k, cd* m);
int gate_nparams(int kind);
bool gate_is_two_qubit(int kind);
qs_status validate_gates(const qs_gate* gates, size_t ngates, int n);

// ---------------------------------------------------------------- fused ops
// Device-independent op after fusion, on *virtual* qubits.
enum FOpType : int { F_G1 = 0, F_G1C = 1, F_D = 2, F_G2 = 3 };

struct FOp {
  FOpType type;
  int t = -1;      // G1/G1C target
  int c = -1;      // G1C choice qubit: matrix m1 when its bit is 1, m0 otherwise
  int a = -1;      // D: first qubit (most significant of the diagonal index); G2: first qubit
  int b = -1;      // D: second qubit or -1 (one-qubit diagonal); G2: second qubit
  cd m0[4], m1[4]; // G1/G1C matrices U[out][in]
  cd d[4];         // D: entries, index 2*bit_a + bit_b (or bit_a when b < 0)
  cd g[16];        // G2 4x4
  int term = -1;   // adjoint sweep: derivative-term slot (the op's matrix is dU/dt U^dagger, not applied)
};

// Converts gates into fused ops.  vmap_out[q] = virtual qubit that holds logical
// qubit q at the end (SWAPs become relabelings).
// fuse: merge one-qubit runs and fold diagonals; relabel: SWAPs become
// relabelings (else they are dense two-qubit ops).
void build_fused_ops(const qs_gate* gates, size_t ngates, int n, std::vector<FOp>& out,
                     std::vector<int>& vmap_out, bool fuse, bool relabel);

// ---------------------------------------------------------------- device ops
template <typename R>
struct alignas(2 * sizeof(R)) C2 {
  R x, y;
};

// kinds of a tile op
// TK_G2: dense 4x4 on qubits a (csrc, cbit) and b (dsrc, dbit), each CS_LANE or
// CS_REG; entries 0..7 in m0, m1, entries 8..15 in the next op (TK_G2C)
enum : uint8_t { TK_REG = 0, TK_LANE = 1, TK_DIAG = 2, TK_G2 = 3, TK_G2C = 4 };
// sources of a choice / diagonal bit
enum : uint8_t { CS_NONE = 0, CS_TILE = 1, CS_LANE = 2, CS_WARP = 3, CS_REG = 4, CS_ONE = 5 };

template <typename R>
struct alignas(16) TileOp {
  uint8_t kind;    // TK_*
  uint8_t slot;    // register slot (TK_REG) or lane bit (TK_LANE)
  uint8_t csrc;    // choice source (TK_REG/TK_LANE) or source of diag bit a (TK_DIAG)
  uint8_t cbit;
  uint8_t dsrc;    // TK_DIAG: source of bit b (CS_NONE for one-qubit diagonals)
  uint8_t dbit;
  int16_t term;    // adjoint pass: index of the derivative term this op forms, or -1
  uint8_t pad[8];
  C2<R> m0[4];     // matrix (choice bit 0) or diagonal d[0..3]
  C2<R> m1[4];     // matrix (choice bit 1)
};

constexpr int kTileBits = 12;     // 4096 amplitudes per tile
constexpr int kLaneBits = 5;
constexpr int kRegBits = 4;       // 16 amplitudes per thread
constexpr int kWarpBits = 3;      // 8 warps, 256 threads
constexpr int kTileThreads = 1 << (kLaneBits + kWarpBits);

struct TileStage {
  uint8_t reg[kRegBits];    // local bit in register slot k
  uint8_t warp[kWarpBits];  // local bit of warp-id bit k
  uint8_t pad;
  int32_t op_begin, op_end;
};

struct TilePass {
  int32_t n_stages;
  int32_t stage_begin;
  int32_t n_nt;                 // number of non-tile bits
  uint8_t pos[kTileBits];       // physical bit of local bit i (ascending)
  uint8_t nt_pos[48];           // physical bits outside the tile (ascending)
};

// Everything one tile-pass launch reads, passed by value as a kernel parameter
// (constant bank; < 32 KiB): the pass, its stages (op ranges relative to the
// pass) and its ops.  The planner keeps passes within these limits.
constexpr int kMaxTileStages = 48;
template <typename R>
struct TileLimits {
  static constexpr int kMaxOps = sizeof(R) == 4 ? 352 : 196;
};
template <typename R>
struct TileParams {
  TilePass pass;
  TileStage stages[kMaxTileStages];
  TileOp<R> ops[TileLimits<R>::kMaxOps];
  const C2<R>* tabs;            // the pass's run tables (device; forward passes with TK_RUN)
  int32_t n_jobs;               // run prologue jobs (RunJob, tile_cp.h)
  uint8_t jobs[64 * 8];
};

// Device-side plain op (one launch per op; also the small-state kernel's op).
template <typename R>
struct alignas(16) PlainOp {
  int32_t type;    // FOpType
  int32_t t, c, a, b;
  int32_t pad[3];
  C2<R> m[16];     // G1: m[0..3]; G1C: m[0..3] choice 0, m[4..7] choice 1; D: m[0..3]; G2: m[0..15]
};

// ---------------------------------------------------------------- plan
struct PlanStep {
  enum Kind { TILE, PLAIN, REMAP, SMALL } kind;
  int index;          // TILE: pass index; PLAIN: op index into plain list; REMAP: remap index
};

struct RemapDesc {
  // A permutation of the bit positions pos[0..11] (ascending): the amplitude
  // bit at local position src[j] moves to local position j.  Positions outside
  // the tile are unchanged, so every CTA reads and writes the same addresses.
  int32_t n_t;                  // tile bits (= kTileBits)
  uint8_t pos[kTileBits];       // physical positions of the tile (ascending)
  uint8_t src[kTileBits];       // local source bit of local destination bit j
  int32_t n_nt;
  uint8_t nt_pos[48];
};

struct Plan {
  std::vector<TilePass> passes;
  std::vector<TileStage> stages;
  std::vector<FOp> tile_fops;       // ops in tile order (converted per precision later)
  std::vector<uint8_t> tile_kind, tile_slot, tile_csrc, tile_cbit, tile_dsrc, tile_dbit;
  std::vector<FOp> plain_fops;      // plain-kernel ops (physical qubit ids)
  std::vector<RemapDesc> remaps;
  std::vector<PlanStep> steps;
  int64_t n_ops = 0;
};

// Plans tile passes for n >= kTileBits.  Ops refer to virtual qubits; l2p maps
// virtual -> physical (updated by remaps); final layout is canonical
// (physical position q holds logical qubit q).
void plan_circuit(const std::vector<FOp>& ops, int n, const std::vector<int>& vmap_final,
                  Plan& plan, int max_ops_per_pass, int max_stages_per_pass);

// ---------------------------------------------------------------- 5-qubit blocks (block_tc.cu)
struct Block {
  int q[5];              // qubits (bit positions); q[i] is bit i of the block's local index
  std::vector<cd> U;     // 32x32 row-major, U[out][in]
  int ngates = 0;
  std::vector<size_t> gate_idx;   // the gates it absorbed (indices into the circuit, in order)
};
// entries of a block with |U_ij| > 0 (dense: more than half of the 1024)
int block_nonzeros(const Block& b);
// Greedy frontier fusion of the circuit into 5-qubit blocks (n >= 5).
void plan_blocks(const qs_gate* gates, size_t ngates, int n, std::vector<Block>& out);
// Tile of a block pass: 12 positions = 5 block qubits + 7 row qubits; the
// tables map an element's "address-order" index (its 12 tile bits sorted by
// physical position, split 6 + 6) to its address offset, row m and column c.
struct BlockPass {
  uint64_t addr_lo[64];
  uint64_t addr_hi[64];
  uint8_t m_lo[64], m_hi[64];
  uint8_t c_lo[64], c_hi[64];
  uint8_t nt_pos[48];           // physical positions outside the tile (ascending)
  int32_t n_nt;
  int32_t flags;                // bit 0: the block is unitary (rows keep their norm);
                                // bit 1: the output goes back by tensor stores (box layout)
  int32_t pad[2];
  // Tile loads as tensor boxes: the 5 tile positions above bit 6 (H, ascending)
  // hold a longest run of g consecutive positions starting at position g_lo (run
  // bits g0 .. g0+g-1 of the run index j = address-order bits 7..11); each of
  // the n_copy = 2^(5-g) copies loads 128 x 2^g amplitudes (bits 0..6 and the
  // run) for one value q of the other H bits, q_off[q] = their address bits.
  // Run j lands in shared-memory slot run_slot[j] (the run's bits lowest).
  uint64_t q_off[16];
  uint8_t run_slot[32];
  // Output staging: row m, column c at m*32 + (c ^ F(m)), F XOR-linear with
  // F(2^j) = stage_f[j]; chosen so that the epilogue's staging writes (a warp's
  // lanes = row bits 0..4) and its reads in address order (a warp's lanes =
  // physical bits 0..4) each fall on 16 distinct 8-byte bank pairs.
  uint8_t stage_f[8];
  int32_t n_copy, g_lo, g_len, g0;
};
void block_pass_desc(int n, const int* bpos, BlockPass& P);
bool block_pass_runs_contiguous(const BlockPass& P);
// U^dagger U = I within 1e-10 (32x32, row-major)
bool block_is_unitary(const cd* U);
size_t block_pass_bytes();
void block_b_operand(const cd* U, int mode, std::vector<unsigned char>& out);
size_t block_b_bytes(int mode);
qs_status launch_block_pass(State* st, const BlockPass& host_pass, const void* pass_dev,
                            const void* b_dev, int mode, int* status_dev);

// ---------------------------------------------------------------- PTM checks (ptm_check.cpp)
// Tolerance of the opt-in channel checks: |G_0j - delta_0j| and the most negative
// Choi eigenvalue allowed.
constexpr double kPtmTol = 1e-8;
double ptm_tp_deviation(const double* G, int n);
double ptm_choi_min_eigenvalue(const double* G, int n);
// Host arrays of count n-qubit PTMs (4^n x 4^n, row-major): QS_EINVAL naming the
// first matrix that is not trace preserving or not completely positive.
qs_status ptm_validate(const double* ptms, int n, int count, const char* what, int* bad_index);

// SMs that block passes leave free while persistent packed kernels of servers
// may run (serve.cu)
int reserved_sms();

// Applies gates to a state (the body of sv_apply_circuit; api.cpp).
qs_status apply_gates(State* st, const qs_gate* gates, size_t ngates, int method, qs_stats* stats,
                      int flags = 0);

// ---------------------------------------------------------------- launchers
// (sv_kernels.cu)
qs_status launch_set_basis(State* st, uint64_t J);
// params: host pointer to a TileParams<float> / TileParams<double> (by value to the kernel)
qs_status launch_tile_pass(State* st, const void* params);
// The adjoint sweep over gates [g0, g1) in fused tile passes: on entry st->data is
// the state after gate g1 - 1 and lam the adjoint state there; on return both are
// the states before gate g0 and dth[3 g + p] has gained dL/dt_p of each gate g in
// the range.  QS_EUNSUPPORTED (nothing launched) for n < 12 or a derivative
// matrix that is not a one-qubit or diagonal op.  Synchronises the stream.
qs_status adjoint_tiled(State* st, void* lam, const qs_gate* gates, size_t g0, size_t g1, double* dth);
// adjoint sweep over one tile pass: st->data = psi, lam the adjoint state, params
// a TileParams image whose ops carry term indices; partial: tiles x nterm values
// in the state's precision
qs_status launch_adjoint_pass(State* st, void* lam, const void* params, void* partial, int nterm);
// dth[slots[i]] += 2 sum over tiles of partial[tile][i]
qs_status launch_term_reduce(State* st, const void* partial, int nterm, const int* slots, double* dth);
qs_status launch_plain_op(State* st, const void* op_dev, int type);
qs_status launch_small(State* st, const void* ops_dev, int nops);
qs_status launch_remap(State* st, const RemapDesc& desc);
qs_status launch_probs(State* st, void* out, int out_fp64, uint64_t mask, double* partials,
                       uint8_t* bits_dev, double* marg_acc);
// probabilities of amplitudes [off, off + count) of the state into out (device;
// float or double), block partial sums of that range into partials
qs_status launch_probs_range(State* st, uint64_t off, uint64_t count, void* out, int out_fp64,
                             double* partials);
qs_status launch_reduce_partials(State* st, const double* partials, int count, double* out);
qs_status launch_loglik(State* st, const uint32_t* counts, double* partials,
                        unsigned long long* clamps);

}  // namespace qs

// The opaque handle of the C ABI is the runtime's State.
struct qs_state_s : public qs::State {};
