// C ABI entry points of the state-vector path (see include/qsim.h).
#include <cstdarg>
#include <cstdio>
#include <complex>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <unordered_map>
#include <utility>

#include "abi_guard.h"
#include "auto_plan.h"
#include "fuse_merge.h"
#include "host_par.h"
#include "internal.h"
#include "tile_cp.h"

namespace qs {

namespace {
thread_local std::string g_err;
}

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

qs_status cuda_status(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return QS_ENOMEM;
  }
  return QS_ECUDA;
}

void* dev_alloc(State* st, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (st->has_alloc) return st->alloc.alloc(bytes, (void*)st->stream, st->alloc.ctx);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(State* st, void* p, size_t bytes) {
  if (!p) return;
  if (st->has_alloc) st->alloc.free(p, bytes, (void*)st->stream, st->alloc.ctx);
  else cudaFree(p);
}

qs_status ensure_opbuf(State* st, size_t bytes) {
  if (bytes <= st->opbuf_bytes) return QS_OK;
  size_t want = 64 * 1024;
  while (want < bytes) want *= 2;
  // the old buffer may still be read by queued kernels
  QS_CUDA(cudaStreamSynchronize(st->stream));
  dev_free(st, st->opbuf, st->opbuf_bytes);
  st->opbuf = dev_alloc(st, want);
  if (!st->opbuf) {
    st->opbuf_bytes = 0;
    set_error("device allocation of %zu bytes for op descriptors failed", want);
    return QS_ENOMEM;
  }
  st->opbuf_bytes = want;
  return QS_OK;
}

// staging of op descriptors: host (pinned) -> device in one copy
qs_status upload(State* st, const std::vector<unsigned char>& blob) {
  if (blob.empty()) return QS_OK;
  qs_status s = ensure_opbuf(st, blob.size());
  if (s != QS_OK) return s;
  if (st->hostbuf_bytes < blob.size()) {
    if (st->hostbuf) {
      QS_CUDA(cudaEventSynchronize(st->upload_done));
      cudaFreeHost(st->hostbuf);
    }
    size_t want = 64 * 1024;
    while (want < blob.size()) want *= 2;
    if (cudaMallocHost(&st->hostbuf, want) != cudaSuccess) {
      cudaGetLastError();
      st->hostbuf = nullptr;
      st->hostbuf_bytes = 0;
      set_error("pinned host allocation failed");
      return QS_ENOMEM;
    }
    st->hostbuf_bytes = want;
  } else {
    QS_CUDA(cudaEventSynchronize(st->upload_done));   // previous copy has read the buffer
  }
  std::memcpy(st->hostbuf, blob.data(), blob.size());
  QS_CUDA(cudaMemcpyAsync(st->opbuf, st->hostbuf, blob.size(), cudaMemcpyHostToDevice, st->stream));
  QS_CUDA(cudaEventRecord(st->upload_done, st->stream));
  return QS_OK;
}

namespace {

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <typename R>
C2<R> c2(cd z) {
  C2<R> r;
  r.x = (R)z.real();
  r.y = (R)z.imag();
  return r;
}

template <typename R>
PlainOp<R> to_plain(const FOp& o) {
  PlainOp<R> p;
  std::memset(&p, 0, sizeof(p));
  p.type = o.type;
  p.t = o.t;
  p.c = o.c;
  p.a = o.a;
  p.b = o.b;
  switch (o.type) {
    case F_G1:
      for (int i = 0; i < 4; ++i) p.m[i] = c2<R>(o.m0[i]);
      break;
    case F_G1C:
      for (int i = 0; i < 4; ++i) {
        p.m[i] = c2<R>(o.m0[i]);
        p.m[4 + i] = c2<R>(o.m1[i]);
      }
      break;
    case F_D:
      for (int i = 0; i < 4; ++i) p.m[i] = c2<R>(o.d[i]);
      break;
    default:
      for (int i = 0; i < 16; ++i) p.m[i] = c2<R>(o.g[i]);
  }
  return p;
}

template <typename R>
TileOp<R> to_tile(const Plan& pl, size_t i) {
  TileOp<R> t;
  std::memset(&t, 0, sizeof(t));
  const FOp& o = pl.tile_fops[i];
  t.kind = pl.tile_kind[i];
  t.slot = pl.tile_slot[i];
  t.csrc = pl.tile_csrc[i];
  t.cbit = pl.tile_cbit[i];
  t.dsrc = pl.tile_dsrc[i];
  t.dbit = pl.tile_dbit[i];
  if (t.kind == TK_G2 || t.kind == TK_G2C) {   // row-major 4x4: entries 0..7, then 8..15
    // canonical order (the kernel has no other variants): register slots ascending,
    // a lane qubit first; swapping a and b swaps the two bits of the local index
    const bool swap = (t.csrc == CS_REG && t.dsrc == CS_REG && t.cbit > t.dbit) ||
                      (t.csrc == CS_REG && t.dsrc == CS_LANE);
    cd G[16];
    for (int l = 0; l < 4; ++l)
      for (int m = 0; m < 4; ++m) {
        const int ls = swap ? ((l & 1) << 1) | (l >> 1) : l, ms = swap ? ((m & 1) << 1) | (m >> 1) : m;
        G[4 * ls + ms] = o.g[4 * l + m];
      }
    if (swap) {
      std::swap(t.csrc, t.dsrc);
      std::swap(t.cbit, t.dbit);
    }
    const int base = t.kind == TK_G2 ? 0 : 8;
    for (int k = 0; k < 4; ++k) {
      t.m0[k] = c2<R>(G[base + k]);
      t.m1[k] = c2<R>(G[base + 4 + k]);
    }
  } else if (o.type == F_D) {
    for (int k = 0; k < 4; ++k) t.m0[k] = c2<R>(o.d[k]);
  } else {
    for (int k = 0; k < 4; ++k) {
      t.m0[k] = c2<R>(o.m0[k]);
      t.m1[k] = c2<R>(o.type == F_G1C ? o.m1[k] : o.m0[k]);
    }
  }
  return t;
}

// A diagonal whose entries are all exactly 1 but the last (a controlled phase,
// or a one-qubit phase) becomes TK_CP: its phase and the context-word positions
// of its bits (see TK_CP); other ops are returned unchanged.
template <typename R>
TileOp<R> cp_form(TileOp<R> t) {
  if (t.kind != TK_DIAG) return t;
  const bool two = t.dsrc != CS_NONE;
  const int last = two ? 3 : 1;
  for (int k = 0; k < last; ++k)
    if (t.m0[k].x != R(1) || t.m0[k].y != R(0)) return t;
  auto ctx_pos = [](uint8_t src, uint8_t bit) -> int {
    switch (src) {
      case CS_TILE: return bit < kCtxOne ? bit : -1;
      case CS_LANE: return kCtxLane + bit;
      case CS_WARP: return kCtxWarp + bit;
      case CS_REG: return 0;   // (not read)
      default: return -1;
    }
  };
  const int pa = ctx_pos(t.csrc, t.cbit), pb = two ? ctx_pos(t.dsrc, t.dbit) : kCtxOne;
  if (pa < 0 || pb < 0) return t;
  const C2<R> p = t.m0[last];
  t.kind = TK_CP;
  t.m0[0] = p;
  for (int k = 1; k < 4; ++k) t.m0[k] = C2<R>{R(0), R(0)};
  t.pad[0] = (uint8_t)pa;
  t.pad[1] = (uint8_t)pb;
  return t;
}

// Packs a run [i, j) of TK_CP ops into a TK_RUN header and its entries (see
// tile_cp.h) at out[w..]; returns the next write index.
template <typename R>
int pack_run(const std::vector<TileOp<R>>& ops, size_t i, size_t j, TileOp<R>* out, int w,
             std::vector<C2<R>>& tabs, std::vector<RunJob>& jobs) {
  using cd = std::complex<double>;
  // context positions: 0 tile bit (the same for the whole CTA), 1 the constant
  // one, 2 a lane or warp bit; bit value of a non-tile position for (lane, warp)
  auto cls = [](int pos) { return pos < kCtxOne ? 0 : (pos == kCtxOne ? 1 : 2); };
  auto bit = [](int pos, int lw) -> int {
    if (pos == kCtxOne) return 1;
    if (pos < kCtxWarp) return ((lw & 31) >> (pos - kCtxLane)) & 1;
    return ((lw >> 5) >> (pos - kCtxWarp)) & 1;
  };
  std::vector<RunEntry<R>> res_s, res_f[4], job_s, job_f[4];
  std::vector<cd> S, N[4], RR;
  auto ones = [](std::vector<cd>& t, size_t n) {
    if (t.empty()) t.assign(n, cd(1.0, 0.0));
  };
  for (size_t o = i; o < j; ++o) {
    const TileOp<R>& t = ops[o];
    RunEntry<R> e;
    std::memset(&e, 0, sizeof(e));
    e.p = t.m0[0];
    const cd p((double)t.m0[0].x, (double)t.m0[0].y);
    const bool ra = t.csrc == CS_REG, rb = t.dsrc == CS_REG;
    if (ra && rb) {
      ones(RR, 16);
      for (int r = 0; r < 16; ++r)
        if ((r >> t.cbit) & (r >> t.dbit) & 1) RR[r] *= p;
    } else if (ra || rb) {   // register slot k; the other bit decides
      const int k = ra ? t.cbit : t.dbit, pa = ra ? t.pad[1] : t.pad[0];
      if (cls(pa) != 0) {
        ones(N[k], kRunTable);
        for (int lw = 0; lw < kRunTable; ++lw)
          if (bit(pa, lw)) N[k][lw] *= p;
      } else {
        e.pa = (uint8_t)pa;
        job_f[k].push_back(e);
      }
    } else {
      const int pa = t.pad[0], pb = t.pad[1];
      e.pa = (uint8_t)pa;
      e.pb = (uint8_t)pb;
      if (cls(pa) != 0 && cls(pb) != 0) {
        ones(S, kRunTable);
        for (int lw = 0; lw < kRunTable; ++lw)
          if (bit(pa, lw) & bit(pb, lw)) S[lw] *= p;
      } else if (cls(pa) != 2 && cls(pb) != 2) {
        job_s.push_back(e);
      } else {
        res_s.push_back(e);
      }
    }
  }
  // prologue jobs while they fit; the rest go to the per-thread lists
  size_t need = !job_s.empty();
  for (int k = 0; k < 4; ++k) need += !job_f[k].empty();
  if (jobs.size() + need > (size_t)kMaxRunJobs) {
    res_s.insert(res_s.end(), job_s.begin(), job_s.end());
    job_s.clear();
    for (int k = 0; k < 4; ++k) {
      res_f[k].insert(res_f[k].end(), job_f[k].begin(), job_f[k].end());
      job_f[k].clear();
    }
  }
  RunHeader rh;
  std::memset(&rh, 0, sizeof(rh));
  rh.n_s = (uint16_t)res_s.size();
  for (int k = 0; k < 4; ++k) rh.n_f[k] = (uint16_t)res_f[k].size();
  rh.ubase = (uint16_t)jobs.size();
  std::vector<RunEntry<R>> all(res_s);
  for (int k = 0; k < 4; ++k) all.insert(all.end(), res_f[k].begin(), res_f[k].end());
  auto add_job = [&](std::vector<RunEntry<R>>& list, bool scalar, int bitno) {
    if (list.empty()) return;
    RunJob jb;
    std::memset(&jb, 0, sizeof(jb));
    jb.op = (uint16_t)w;
    jb.first = (uint16_t)all.size();
    jb.count = (uint16_t)list.size();
    jb.scalar = scalar ? 1 : 0;
    jobs.push_back(jb);
    rh.umask |= (uint8_t)(1u << bitno);
    all.insert(all.end(), list.begin(), list.end());
  };
  add_job(job_s, true, 0);
  for (int k = 0; k < 4; ++k) add_job(job_f[k], false, 1 + k);
  rh.toff = (uint32_t)tabs.size();
  auto add_tab = [&](const std::vector<cd>& t, int bitno) {
    if (t.empty()) return;
    rh.tmask |= (uint8_t)(1u << bitno);
    for (const cd& x : t) tabs.push_back(C2<R>{(R)x.real(), (R)x.imag()});
  };
  add_tab(S, 0);
  for (int k = 0; k < 4; ++k) add_tab(N[k], 1 + k);
  add_tab(RR, 5);
  TileOp<R> h;
  std::memset(&h, 0, sizeof(h));
  h.kind = TK_RUN;
  static_assert(sizeof(RunHeader) <= sizeof(h.m0), "run header fits the op's matrix");
  std::memcpy(&h.m0[0], &rh, sizeof(rh));
  const size_t per = sizeof(TileOp<R>) / sizeof(RunEntry<R>);
  const size_t nslots = (all.size() + per - 1) / per;
  h.slot = (uint8_t)nslots;
  out[w++] = h;
  std::vector<TileOp<R>> slots(nslots);
  std::memset(slots.data(), 0, sizeof(TileOp<R>) * nslots);
  if (!all.empty()) std::memcpy((void*)slots.data(), all.data(), sizeof(RunEntry<R>) * all.size());
  for (size_t k = 0; k < nslots; ++k) out[w++] = slots[k];
  return w;
}

// The kernel-parameter image of one forward tile pass: ops converted per
// precision, controlled phases in their TK_CP form, and runs of at least kRunMin
// of them packed into TK_RUN entry lists and tables (at most 255 op slots each, 5
// entries per slot for complex64); stage op ranges relative to the pass.  tabs
// receives the pass's run tables (offsets relative to its start).
constexpr size_t kRunMin = 3;
template <typename R>
void build_pass_params(const Plan& pl, const TilePass& pass, TileParams<R>* tp, std::vector<C2<R>>& tabs) {
  std::memset(tp, 0, sizeof(TileParams<R>));
  tp->pass = pass;
  tp->pass.stage_begin = 0;
  tabs.clear();
  std::vector<RunJob> jobs;
  int w = 0;
  std::vector<TileOp<R>> conv;
  const size_t per = sizeof(TileOp<R>) / sizeof(RunEntry<R>);
  for (int s2 = 0; s2 < pass.n_stages; ++s2) {
    TileStage ts = pl.stages[pass.stage_begin + s2];
    conv.clear();
    for (int o = ts.op_begin; o < ts.op_end; ++o) conv.push_back(cp_form(to_tile<R>(pl, (size_t)o)));
    ts.op_begin = w;
    for (size_t i = 0; i < conv.size();) {
      if (conv[i].kind == TK_CP) {
        size_t j = i;
        while (j < conv.size() && conv[j].kind == TK_CP && j - i < 255 * per) ++j;
        if (j - i >= kRunMin) {
          w = pack_run(conv, i, j, tp->ops, w, tabs, jobs);
          i = j;
          continue;
        }
      }
      tp->ops[w++] = conv[i++];
    }
    ts.op_end = w;
    tp->stages[s2] = ts;
  }
  tp->n_jobs = (int32_t)jobs.size();
  static_assert(sizeof(tp->jobs) >= sizeof(RunJob) * kMaxRunJobs, "job table fits");
  if (!jobs.empty()) std::memcpy(tp->jobs, jobs.data(), sizeof(RunJob) * jobs.size());
}

template <typename T>
size_t put(std::vector<unsigned char>& blob, const T* p, size_t count) {
  size_t off = align16(blob.size());
  blob.resize(off + sizeof(T) * count);
  if (count) std::memcpy(blob.data() + off, p, sizeof(T) * count);
  return off;
}

// algorithmic flops per amplitude of a fused op (2 per real FMA of its complex MACs)
double op_flops_per_amp(const FOp& o) {
  switch (o.type) {
    case F_G1: case F_G1C: return 16.0;
    case F_D: return 8.0;
    default: return 32.0;
  }
}

// Process-wide profiling session (qs_profile_begin / qs_profile_end).
struct ProfileSession {
  std::mutex mu;
  bool active = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;
};
ProfileSession& profile() {
  static ProfileSession p;
  return p;
}

// Optional CUDA-event timing of every launch, by kind (tile, plain, remap, small):
// per call (QS_OPT_TIME_KERNELS) and/or into the profiling session.
struct KernelTimer {
  bool on = false;
  cudaStream_t stream = nullptr;
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;
  cudaEvent_t prof_start = nullptr;
  void before(int k) {
    ProfileSession& ps = profile();
    if (ps.active) {
      std::lock_guard<std::mutex> g(ps.mu);
      cudaEvent_t a;
      cudaEventCreate(&a);
      cudaEventRecord(a, stream);
      ps.ev.push_back(a);
      ps.ev.push_back(nullptr);
      ps.kind.push_back(k);
      prof_start = a;
    }
    if (!on) return;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, stream);
    ev.push_back(a);
    ev.push_back(b);
    kind.push_back(k);
  }
  void after() {
    ProfileSession& ps = profile();
    if (ps.active && prof_start) {
      std::lock_guard<std::mutex> g(ps.mu);
      cudaEvent_t b;
      cudaEventCreate(&b);
      cudaEventRecord(b, stream);
      for (size_t i = ps.ev.size(); i >= 2; i -= 2)
        if (ps.ev[i - 2] == prof_start) {
          ps.ev[i - 1] = b;
          break;
        }
      prof_start = nullptr;
    }
    if (on) cudaEventRecord(ev.back(), stream);
  }
  void finish(qs_stats* stats) {
    if (!on) return;
    cudaStreamSynchronize(stream);
    for (size_t i = 0; i < kind.size(); ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
      if (stats) stats->kernel_ms[kind[i]] += ms;
      cudaEventDestroy(ev[2 * i]);
      cudaEventDestroy(ev[2 * i + 1]);
    }
    ev.clear();
    kind.clear();
  }
};

template <typename R>
qs_status run_plain(State* st, const std::vector<FOp>& fops, qs_stats* stats, KernelTimer& tm) {
  double flops = 0.0;
  for (const FOp& o : fops) {
    PlainOp<R> p = to_plain<R>(o);
    tm.before(1);
    qs_status s = launch_plain_op(st, &p, o.type);
    tm.after();
    if (s != QS_OK) return s;
    flops += op_flops_per_amp(o) * std::ldexp(1.0, st->n);
  }
  if (stats) {
    stats->ops_fused = (int64_t)fops.size();
    stats->passes = (int64_t)fops.size();
    stats->launches = (int64_t)fops.size();
    stats->flops = flops;
  }
  return QS_OK;
}

template <typename R>
qs_status run_small(State* st, const std::vector<FOp>& fops, qs_stats* stats, KernelTimer& tm) {
  std::vector<PlainOp<R>> ops;
  ops.reserve(fops.size());
  double flops = 0.0;
  for (const FOp& o : fops) {
    ops.push_back(to_plain<R>(o));
    flops += op_flops_per_amp(o) * std::ldexp(1.0, st->n);
  }
  std::vector<unsigned char> blob;
  size_t off = put(blob, ops.data(), ops.size());
  qs_status s = upload(st, blob);
  if (s != QS_OK) return s;
  tm.before(3);
  s = launch_small(st, (unsigned char*)st->opbuf + off, (int)ops.size());
  tm.after();
  if (s != QS_OK) return s;
  if (stats) {
    stats->ops_fused = (int64_t)fops.size();
    stats->passes = 1;
    stats->launches = 1;
    stats->flops = flops;
    stats->upload_bytes = (int64_t)blob.size();
  }
  return QS_OK;
}

template <typename R>
qs_status run_tiled(State* st, const std::vector<FOp>& fops, const std::vector<int>& vmap,
                    qs_stats* stats, KernelTimer& tm) {
  Plan pl;
  plan_circuit(fops, st->n, vmap, pl, TileLimits<R>::kMaxOps, kMaxTileStages);
  std::vector<unsigned char> blob;
  // every pass's kernel-parameter image first, its run tables into the upload
  // (remap descriptors go by value as kernel parameters)
  std::vector<TileParams<R>> tps;
  std::vector<size_t> tab_off;
  {
    size_t ntile = 0;
    for (const PlanStep& step : pl.steps) ntile += step.kind == PlanStep::TILE;
    tps.resize(ntile);
    std::vector<C2<R>> tabs;
    size_t ti = 0;
    for (const PlanStep& step : pl.steps) {
      if (step.kind != PlanStep::TILE) continue;
      build_pass_params<R>(pl, pl.passes[step.index], &tps[ti++], tabs);
      tab_off.push_back(tabs.empty() ? SIZE_MAX : put(blob, tabs.data(), tabs.size()));
    }
  }
  qs_status s = upload(st, blob);
  if (s != QS_OK) return s;
  unsigned char* dev = (unsigned char*)st->opbuf;
  int64_t passes = 0, launches = 0, tile_launches = 0;
  const double N = std::ldexp(1.0, st->n);
  double tile_flops = 0.0, plain_flops = 0.0;
  for (size_t i = 0; i < pl.tile_fops.size(); ++i)   // a dense two-qubit op has two entries
    if (pl.tile_kind[i] != TK_G2C) tile_flops += op_flops_per_amp(pl.tile_fops[i]) * N;
  size_t ti = 0;
  for (const PlanStep& step : pl.steps) {
    switch (step.kind) {
      case PlanStep::TILE: {
        TileParams<R>& tp = tps[ti];
        tp.tabs = tab_off[ti] == SIZE_MAX ? nullptr : (const C2<R>*)(dev + tab_off[ti]);
        ++ti;
        tm.before(0);
        s = launch_tile_pass(st, &tp);
        ++tile_launches;
        break;
      }
      case PlanStep::PLAIN: {
        PlainOp<R> p = to_plain<R>(pl.plain_fops[step.index]);
        plain_flops += op_flops_per_amp(pl.plain_fops[step.index]) * N;
        tm.before(1);
        s = launch_plain_op(st, &p, p.type);
        break;
      }
      case PlanStep::REMAP:
        tm.before(2);
        s = launch_remap(st, pl.remaps[step.index]);
        break;
      default:
        break;
    }
    tm.after();
    if (s != QS_OK) return s;
    ++passes;
    ++launches;
  }
  if (stats) {
    stats->ops_fused = (int64_t)fops.size();
    stats->passes = passes;
    stats->launches = launches;
    stats->tile_launches = tile_launches;
    stats->tile_flops = tile_flops;
    stats->flops = tile_flops + plain_flops;
    stats->upload_bytes = (int64_t)blob.size();
  }
  return QS_OK;
}

// The adjoint sweep over gates [g0, g1) fused into tile passes.  The reversed
// gate list becomes, per gate, one op per parameter carrying its derivative
// matrix G_p = (dU/dt_p) U^dagger (a term op, not applied) followed by
// U^dagger; the tile planner splits it into passes (an op keeps its order with
// the ops that share a qubit), and each pass runs the adjoint pass kernel on
// psi = st->data and lam, its per-tile terms reduced into dth.  Dense two-qubit
// U^dagger ops (SWAP, MAT2) run as plain launches on both states.
template <typename R>
qs_status adjoint_tiled_t(State* st, void* lam, const qs_gate* gates, size_t g0, size_t g1, double* dth) {
  const int n = st->n;
  if (n < kTileBits) {
    set_error("fused adjoint needs n >= %d", kTileBits);
    return QS_EUNSUPPORTED;
  }
  std::vector<qs_gate> bw;
  std::vector<int> slot;
  for (size_t g = g1; g-- > g0;) {
    const qs_gate& G = gates[g];
    cd U[16], Ud[16];
    int dim = 0;
    gate_matrix(G, U, &dim);
    for (int r = 0; r < dim; ++r)
      for (int c = 0; c < dim; ++c) Ud[r * dim + c] = std::conj(U[c * dim + r]);
    auto as_gate = [&](const cd* m) {
      qs_gate x;
      std::memset(&x, 0, sizeof(x));
      x.kind = dim == 2 ? QS_MAT1 : QS_MAT2;
      x.q[0] = G.q[0];
      x.q[1] = dim == 2 ? 0 : G.q[1];
      for (int i = 0; i < dim * dim; ++i) {
        x.m[2 * i] = m[i].real();
        x.m[2 * i + 1] = m[i].imag();
      }
      return x;
    };
    const int np = gate_nparams(G.kind);
    for (int p = 0; p < np; ++p) {
      cd dU[16], M[16];
      gate_dmatrix(G, p, dU);
      for (int r = 0; r < dim; ++r)
        for (int c = 0; c < dim; ++c) {
          cd acc = 0;
          for (int k = 0; k < dim; ++k) acc += dU[r * dim + k] * Ud[k * dim + c];
          M[r * dim + c] = acc;
        }
      bw.push_back(as_gate(M));
      slot.push_back((int)(3 * g + p));
    }
    bw.push_back(as_gate(Ud));
    slot.push_back(-1);
  }
  std::vector<FOp> fops;
  std::vector<int> vmap;
  build_fused_ops(bw.data(), bw.size(), n, fops, vmap, /*fuse=*/false, /*relabel=*/false);
  if (fops.size() != bw.size()) {
    set_error("adjoint op list changed size");
    return QS_EUNSUPPORTED;
  }
  for (size_t i = 0; i < fops.size(); ++i) {
    fops[i].term = slot[i];
    if (slot[i] >= 0 && fops[i].type != F_G1 && fops[i].type != F_D) {
      set_error("derivative matrix of gate %d is not a one-qubit or diagonal op", slot[i] / 3);
      return QS_EUNSUPPORTED;
    }
  }
  for (int q = 0; q < n; ++q) vmap[q] = q;
  Plan pl;
  plan_circuit(fops, n, vmap, pl, TileLimits<R>::kMaxOps, kMaxTileStages);
  if (!pl.remaps.empty()) {
    set_error("adjoint plan needs a remap");
    return QS_EUNSUPPORTED;
  }
  const uint64_t tiles = 1ull << (n - kTileBits);
  const size_t pbytes = sizeof(R) * tiles * TileLimits<R>::kMaxOps;
  void* partial = dev_alloc(st, pbytes);
  if (!partial) {
    set_error("adjoint partials allocation failed");
    return QS_ENOMEM;
  }
  // the term slots of every pass, uploaded once
  std::vector<int> slots_all;
  std::vector<size_t> slot_off;
  for (const PlanStep& step : pl.steps) {
    slot_off.push_back(slots_all.size());
    if (step.kind != PlanStep::TILE) continue;
    const TilePass& pass = pl.passes[step.index];
    for (int s2 = 0; s2 < pass.n_stages; ++s2) {
      const TileStage& ts = pl.stages[pass.stage_begin + s2];
      for (int o = ts.op_begin; o < ts.op_end; ++o)
        if (pl.tile_fops[o].term >= 0) slots_all.push_back(pl.tile_fops[o].term);
    }
  }
  std::vector<unsigned char> blob;
  const size_t off_slots = put(blob, slots_all.data(), slots_all.size());
  qs_status s = upload(st, blob);
  const int* slots_dev = (const int*)((unsigned char*)st->opbuf + off_slots);
  std::unique_ptr<TileParams<R>> tp(new TileParams<R>());
  for (size_t si = 0; si < pl.steps.size() && s == QS_OK; ++si) {
    const PlanStep& step = pl.steps[si];
    if (step.kind == PlanStep::TILE) {
      const TilePass& pass = pl.passes[step.index];
      std::memset(tp.get(), 0, sizeof(TileParams<R>));
      tp->pass = pass;
      const int op0 = pl.stages[pass.stage_begin].op_begin;
      int nterm = 0;
      for (int s2 = 0; s2 < pass.n_stages; ++s2) {
        TileStage ts = pl.stages[pass.stage_begin + s2];
        for (int o = ts.op_begin; o < ts.op_end; ++o) {
          TileOp<R> t = to_tile<R>(pl, (size_t)o);
          t.term = pl.tile_fops[o].term >= 0 ? (int16_t)nterm++ : (int16_t)-1;
          tp->ops[o - op0] = t;
        }
        ts.op_begin -= op0;
        ts.op_end -= op0;
        tp->stages[s2] = ts;
      }
      tp->pass.stage_begin = 0;
      s = launch_adjoint_pass(st, lam, tp.get(), partial, nterm);
      if (s == QS_OK) s = launch_term_reduce(st, partial, nterm, slots_dev + slot_off[si], dth);
    } else if (step.kind == PlanStep::PLAIN) {
      PlainOp<R> p = to_plain<R>(pl.plain_fops[step.index]);
      s = launch_plain_op(st, &p, p.type);
      void* psi = st->data;
      st->data = lam;
      if (s == QS_OK) s = launch_plain_op(st, &p, p.type);
      st->data = psi;
    } else {
      set_error("unexpected step in the adjoint plan");
      s = QS_EUNSUPPORTED;
    }
  }
  cudaStreamSynchronize(st->stream);
  dev_free(st, partial, pbytes);
  return s;
}

// Dense 5-qubit blocks on the tensor cores: one pass per block.
qs_status run_block_list(State* st, const std::vector<Block>& blocks, int mode, qs_stats* stats,
                         KernelTimer& tm) {
  if (blocks.empty()) return QS_OK;
  std::vector<unsigned char> blob(16, 0);   // status word of the bounded waits
  std::vector<BlockPass> passes(blocks.size());
  for (size_t i = 0; i < blocks.size(); ++i) {
    block_pass_desc(st->n, blocks[i].q, passes[i]);
    if (!block_pass_runs_contiguous(passes[i])) {
      set_error("block pass: tile layout without contiguous low bits");
      return QS_EUNSUPPORTED;
    }
  }
  // per block (independent, on host threads): the unitarity flag and the split B operand
  const size_t bb = block_b_bytes(mode);
  std::vector<unsigned char> bops(bb * blocks.size());
  std::vector<char> unitary(blocks.size(), 0);
  parallel_for(blocks.size(), 4, [&](size_t i) {
    unitary[i] = block_is_unitary(blocks[i].U.data()) ? 1 : 0;
    std::vector<unsigned char> tmp;
    block_b_operand(blocks[i].U.data(), mode, tmp);
    std::memcpy(bops.data() + i * bb, tmp.data(), bb);
  });
  for (size_t i = 0; i < blocks.size(); ++i)
    if (unitary[i]) passes[i].flags |= 1;
  const size_t off_pass = put(blob, passes.data(), passes.size());
  const size_t off_b = align16(blob.size());
  blob.resize(off_b + bops.size());
  std::memcpy(blob.data() + off_b, bops.data(), bops.size());
  qs_status s = upload(st, blob);
  if (s != QS_OK) return s;
  unsigned char* dev = (unsigned char*)st->opbuf;
  int* status_dev = (int*)dev;
  for (size_t i = 0; i < blocks.size(); ++i) {
    tm.before(4);
    s = launch_block_pass(st, passes[i], dev + off_pass + i * sizeof(BlockPass), dev + off_b + i * bb,
                          mode, status_dev);
    tm.after();
    if (s != QS_OK) return s;
  }
  int status = 0;
  QS_CUDA(cudaMemcpyAsync(&status, status_dev, sizeof(int), cudaMemcpyDeviceToHost, st->stream));
  QS_CUDA(cudaStreamSynchronize(st->stream));
  if (status != 0) {
    set_error("block GEMM kernel: bounded wait on the tensor-core barrier gave up");
    return QS_ETIMEOUT;
  }
  if (stats) {
    stats->ops_fused += (int64_t)blocks.size();
    stats->passes += (int64_t)blocks.size();
    stats->launches += (int64_t)blocks.size();
    // 32 complex MACs per amplitude per block = 256 flops (the split precision triples the MMAs)
    stats->flops += 256.0 * std::ldexp(1.0, st->n) * (double)blocks.size();
    stats->upload_bytes += (int64_t)blob.size();
  }
  return QS_OK;
}

qs_status run_blocks(State* st, const qs_gate* gates, size_t ngates, int mode, qs_stats* stats,
                     KernelTimer& tm) {
  std::vector<Block> blocks;
  plan_blocks(gates, ngates, st->n, blocks);
  return run_block_list(st, blocks, mode, stats, tm);
}

// QS_METHOD_AUTO (complex64, n >= 12): the circuit is cut into 5-qubit blocks;
// a dense block (more than half of its 1024 entries nonzero) is a real
// contraction and goes to the tensor cores, and every maximal run of sparse
// blocks (diagonal or nearly diagonal stretches such as the QFT's controlled
// phases) goes back to its gates, which the tile planner fuses into shared-memory
// passes of 12 qubits.  Both kinds of segment start and end in the canonical
// layout, and applying the blocks in order equals the circuit, so the segments
// compose.
qs_status run_auto(State* st, const qs_gate* gates, size_t ngates, qs_stats* stats, KernelTimer& tm) {
  std::vector<Block> blocks;
  plan_blocks(gates, ngates, st->n, blocks);
  // one or two dense blocks among sparse ones (the QFT's Hadamards among its
  // phases) may run on tile passes alone (auto_plan.h)
  {
    std::vector<FOp> fops;
    std::vector<int> vmap;
    if (auto_all_tiles(gates, ngates, st->n, blocks, &fops, &vmap)) {
      qs_stats part;
      std::memset(&part, 0, sizeof(part));
      qs_status s = run_tiled<float>(st, fops, vmap, &part, tm);
      if (stats) {
        stats->ops_fused = part.ops_fused;
        stats->passes = part.passes;
        stats->launches = part.launches;
        stats->tile_launches = part.tile_launches;
        stats->tile_flops = part.tile_flops;
        stats->flops = part.flops;
        stats->upload_bytes = part.upload_bytes;
      }
      if (s == QS_OK) QS_CUDA(cudaStreamSynchronize(st->stream));
      return s;
    }
  }
  size_t i = 0;
  qs_status s = QS_OK;
  while (i < blocks.size() && s == QS_OK) {
    const bool dense = block_nonzeros(blocks[i]) > 512;
    size_t j = i;
    while (j < blocks.size() && (block_nonzeros(blocks[j]) > 512) == dense) ++j;
    if (dense) {
      std::vector<Block> seg(std::make_move_iterator(blocks.begin() + (long)i),
                             std::make_move_iterator(blocks.begin() + (long)j));
      s = run_block_list(st, seg, 1, stats, tm);
    } else {
      std::vector<qs_gate> seg;
      for (size_t k = i; k < j; ++k)
        for (size_t gi : blocks[k].gate_idx) seg.push_back(gates[gi]);
      std::vector<FOp> fops;
      std::vector<int> vmap;
      build_fused_ops(seg.data(), seg.size(), st->n, fops, vmap, /*fuse=*/true, /*relabel=*/true);
      qs_stats part;
      std::memset(&part, 0, sizeof(part));
      s = run_tiled<float>(st, fops, vmap, &part, tm);
      if (stats) {
        stats->ops_fused += part.ops_fused;
        stats->passes += part.passes;
        stats->launches += part.launches;
        stats->tile_launches += part.tile_launches;
        stats->tile_flops += part.tile_flops;
        stats->flops += part.flops;
        stats->upload_bytes += part.upload_bytes;
      }
    }
    i = j;
  }
  if (s == QS_OK) {   // the tile segments run asynchronously; report their faults here too
    QS_CUDA(cudaStreamSynchronize(st->stream));
  }
  return s;
}

qs_status check_state(qs_state_t st) {
  if (!st) {
    set_error("state is NULL");
    return QS_EINVAL;
  }
  return QS_OK;
}

}  // namespace

// The kernel-parameter image of a forward tile pass and its run tables (tile_cp.h).
template <typename R>
void tile_pass_image(const Plan& pl, const TilePass& pass, TileParams<R>* tp, std::vector<C2<R>>& tabs) {
  build_pass_params<R>(pl, pass, tp, tabs);
}
template void tile_pass_image<float>(const Plan&, const TilePass&, TileParams<float>*, std::vector<C2<float>>&);
template void tile_pass_image<double>(const Plan&, const TilePass&, TileParams<double>*, std::vector<C2<double>>&);


qs_status adjoint_tiled(State* st, void* lam, const qs_gate* gates, size_t g0, size_t g1, double* dth) {
  return st->prec == QS_C64 ? adjoint_tiled_t<float>(st, lam, gates, g0, g1, dth)
                            : adjoint_tiled_t<double>(st, lam, gates, g0, g1, dth);
}

qs_status apply_gates(State* st, const qs_gate* gates, size_t ngates, int method, qs_stats* stats,
                      int flags) {
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (method < QS_METHOD_TILED || method > QS_METHOD_AUTO) {
    set_error("unknown method %d", method);
    return QS_EINVAL;
  }
  // AUTO: blocks and tile passes where the state allows the blocks, else tiles
  const bool autom = method == QS_METHOD_AUTO && st->prec == QS_C64 && st->n >= kTileBits;
  if (method == QS_METHOD_AUTO && !autom) method = QS_METHOD_TILED;
  const bool blocks = method == QS_METHOD_BLOCKS_TF32 || method == QS_METHOD_BLOCKS_BF16;
  if (blocks && (st->prec != QS_C64 || st->n < kTileBits)) {
    set_error("the tensor-core block method needs a complex64 state of at least %d qubits", kTileBits);
    return QS_EUNSUPPORTED;
  }
  if (ngates == 0) return QS_OK;
  std::vector<FOp> fops;
  std::vector<int> vmap;
  const bool c64 = st->prec == QS_C64;
  KernelTimer tm;
  tm.on = (flags & QS_OPT_TIME_KERNELS) != 0;
  tm.stream = st->stream;
  qs_status s;
  if (autom) {
    s = run_auto(st, gates, ngates, stats, tm);
  } else if (blocks) {
    s = run_blocks(st, gates, ngates, method == QS_METHOD_BLOCKS_TF32 ? 0 : 1, stats, tm);
  } else if (method == QS_METHOD_PLAIN) {
    build_fused_ops(gates, ngates, st->n, fops, vmap, /*fuse=*/false, /*relabel=*/false);
    s = c64 ? run_plain<float>(st, fops, stats, tm) : run_plain<double>(st, fops, stats, tm);
  } else if (st->n < kTileBits) {
    build_fused_ops(gates, ngates, st->n, fops, vmap, /*fuse=*/true, /*relabel=*/false);
    merge_one_qubit_ops(fops, st->n, nullptr);   // one CTA runs them all: no passes to keep
    s = c64 ? run_small<float>(st, fops, stats, tm) : run_small<double>(st, fops, stats, tm);
  } else {
    build_fused_ops(gates, ngates, st->n, fops, vmap, /*fuse=*/true, /*relabel=*/true);
    s = c64 ? run_tiled<float>(st, fops, vmap, stats, tm)
            : run_tiled<double>(st, fops, vmap, stats, tm);
  }
  tm.finish(stats);
  if (stats) {
    stats->gates_in = (int64_t)ngates;
    stats->bytes_moved = (double)stats->passes * 2.0 * (double)st->data_bytes;
  }
  return s;
}

// Copies of probabilities to host memory queued by sv_probs_host_async, per
// state: two device buffers used in turn, a non-blocking copy stream, and per
// buffer an event when its probabilities are formed (state's stream) and one
// when its copy has ended (copy stream).  Kept beside the state, keyed by it.
struct HostCopies {
  void* buf = nullptr;   // 2 * half bytes
  size_t half = 0;
  cudaStream_t cs = nullptr;
  cudaEvent_t formed[2] = {nullptr, nullptr};
  cudaEvent_t copied[2] = {nullptr, nullptr};
  bool queued[2] = {false, false};
  int next = 0;
};
std::mutex g_copies_mu;
std::unordered_map<const State*, HostCopies*> g_copies;

HostCopies* find_copies(const State* st) {
  std::lock_guard<std::mutex> g(g_copies_mu);
  auto it = g_copies.find(st);
  return it == g_copies.end() ? nullptr : it->second;
}

// waits for the state's queued copies (if any); the first error is returned
qs_status wait_copies(State* st) {
  HostCopies* hc = find_copies(st);
  if (!hc) return QS_OK;
  const cudaError_t e = cudaStreamSynchronize(hc->cs);
  hc->queued[0] = hc->queued[1] = false;
  return e == cudaSuccess ? QS_OK : cuda_status(e, "copy of probabilities to the host");
}

void release_copies(State* st) {
  HostCopies* hc = nullptr;
  {
    std::lock_guard<std::mutex> g(g_copies_mu);
    auto it = g_copies.find(st);
    if (it == g_copies.end()) return;
    hc = it->second;
    g_copies.erase(it);
  }
  if (hc->cs) cudaStreamSynchronize(hc->cs);
  if (hc->buf) dev_free(st, hc->buf, 2 * hc->half);
  for (int k = 0; k < 2; ++k) {
    if (hc->formed[k]) cudaEventDestroy(hc->formed[k]);
    if (hc->copied[k]) cudaEventDestroy(hc->copied[k]);
  }
  if (hc->cs) cudaStreamDestroy(hc->cs);
  delete hc;
}

// the state's copy pipeline with buffers of at least `half` bytes each
qs_status copies_for(State* st, size_t half, HostCopies** out) {
  HostCopies* hc = find_copies(st);
  if (hc && hc->half < half) {   // buffers too small (an fp64 call after fp32 ones): start over
    cudaStreamSynchronize(st->stream);   // no kernel of the state may still write them
    release_copies(st);
    hc = nullptr;
  }
  if (!hc) {
    hc = new (std::nothrow) HostCopies();
    if (!hc) {
      set_error("host copy pipeline: out of host memory");
      return QS_ENOMEM;
    }
    cudaError_t e = cudaStreamCreateWithFlags(&hc->cs, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      e = cudaEventCreateWithFlags(&hc->formed[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hc->copied[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) {
      hc->buf = dev_alloc(st, 2 * half);
      hc->half = half;
    }
    {
      std::lock_guard<std::mutex> g(g_copies_mu);
      g_copies[st] = hc;   // released by release_copies on every path below
    }
    if (e != cudaSuccess) {
      const qs_status s = cuda_status(e, "host copy pipeline");
      release_copies(st);
      return s;
    }
    if (!hc->buf) {
      hc->half = 0;
      release_copies(st);
      set_error("device buffers for the host copies of the probabilities could not be allocated");
      return QS_ENOMEM;
    }
  }
  *out = hc;
  return QS_OK;
}

}  // namespace qs

using namespace qs;

extern "C" {

const char* qs_last_error(void) { return g_err.c_str(); }

const char* qs_version(void) { return "qsim-gb300 0.5 (sm_103a)"; }

qs_status sv_create(int n, int prec, const qs_allocator* alloc, void* stream, qs_state_t* out) {
  return abi_guard(__func__, [&]() -> qs_status {
    if (!out) {
      set_error("out is NULL");
      return QS_EINVAL;
    }
    *out = nullptr;
    if (n < 1 || n > 36) {
      set_error("n = %d outside [1, 36]", n);
      return QS_EINVAL;
    }
    if (prec != QS_C64 && prec != QS_C128) {
      set_error("bad precision %d", prec);
      return QS_EINVAL;
    }
    qs_state_s* st = new (std::nothrow) qs_state_s();
    if (!st) return QS_ENOMEM;
    st->n = n;
    st->prec = prec;
    st->amp_bytes = prec == QS_C64 ? 8 : 16;
    st->stream = (cudaStream_t)stream;
    if (alloc && alloc->alloc && alloc->free) {
      st->alloc = *alloc;
      st->has_alloc = true;
    }
    cudaGetDevice(&st->device);
    st->data_bytes = st->amp_bytes << n;
    st->data = dev_alloc(st, st->data_bytes);
    if (!st->data) {
      set_error("device allocation of %zu bytes for a %d-qubit state failed", st->data_bytes, n);
      delete st;
      return QS_ENOMEM;
    }
    st->scratch_bytes = kScratchBytes;
    st->scratch = dev_alloc(st, st->scratch_bytes);
    if (!st->scratch) {
      dev_free(st, st->data, st->data_bytes);
      set_error("scratch allocation failed");
      delete st;
      return QS_ENOMEM;
    }
    if (cudaEventCreateWithFlags(&st->upload_done, cudaEventDisableTiming) != cudaSuccess) {
      dev_free(st, st->scratch, st->scratch_bytes);
      dev_free(st, st->data, st->data_bytes);
      qs_status s = cuda_status(cudaGetLastError(), "cudaEventCreate");
      delete st;
      return s;
    }
    qs_status s = launch_set_basis(st, 0);
    if (s != QS_OK) {
      sv_destroy(st);
      return s;
    }
    *out = st;
    return QS_OK;
  });
}

qs_status sv_wrap(int n, int prec, void* device_buf, const qs_allocator* alloc, void* stream, qs_state_t* out) {
  return abi_guard(__func__, [&]() -> qs_status {
    if (!out || !device_buf) {
      set_error("out and device_buf are required");
      return QS_EINVAL;
    }
    *out = nullptr;
    if (n < 1 || n > 36 || (prec != QS_C64 && prec != QS_C128)) {
      set_error("n = %d outside [1, 36] or bad precision %d", n, prec);
      return QS_EINVAL;
    }
    if ((uintptr_t)device_buf & 15) {
      set_error("device_buf must be 16-byte aligned");
      return QS_EINVAL;
    }
    qs_state_s* st = new (std::nothrow) qs_state_s();
    if (!st) return QS_ENOMEM;
    st->n = n;
    st->prec = prec;
    st->amp_bytes = prec == QS_C64 ? 8 : 16;
    st->stream = (cudaStream_t)stream;
    if (alloc && alloc->alloc && alloc->free) {
      st->alloc = *alloc;
      st->has_alloc = true;
    }
    cudaGetDevice(&st->device);
    st->data_bytes = st->amp_bytes << n;
    st->data = device_buf;
    st->owns_data = false;
    st->scratch_bytes = kScratchBytes;
    st->scratch = dev_alloc(st, st->scratch_bytes);
    if (!st->scratch) {
      set_error("scratch allocation failed");
      delete st;
      return QS_ENOMEM;
    }
    if (cudaEventCreateWithFlags(&st->upload_done, cudaEventDisableTiming) != cudaSuccess) {
      dev_free(st, st->scratch, st->scratch_bytes);
      qs_status s = cuda_status(cudaGetLastError(), "cudaEventCreate");
      delete st;
      return s;
    }
    *out = st;
    return QS_OK;
  });
}

qs_status sv_destroy(qs_state_t st) {
  return abi_guard(__func__, [&]() -> qs_status {
    if (!st) return QS_OK;
    cudaStreamSynchronize(st->stream);
    release_copies(st);
    dev_free(st, st->opbuf, st->opbuf_bytes);
    if (st->stage) dev_free(st, st->stage, st->stage_bytes);
    dev_free(st, st->scratch, st->scratch_bytes);
    if (st->owns_data) dev_free(st, st->data, st->data_bytes);
    if (st->hostbuf) cudaFreeHost(st->hostbuf);
    if (st->upload_done) cudaEventDestroy(st->upload_done);
    delete st;
    return QS_OK;
  });
}

qs_status sv_set_stream(qs_state_t st, void* stream) {
  return abi_guard(__func__, [&]() -> qs_status {
    qs_status s = check_state(st);
    if (s != QS_OK) return s;
    QS_CUDA(cudaStreamSynchronize(st->stream));
    st->stream = (cudaStream_t)stream;
    return QS_OK;
  });
}

qs_status sv_info(qs_state_t st, int* n, int* prec, void** device_ptr) {
  return abi_guard(__func__, [&]() -> qs_status {
    qs_status s = check_state(st);
    if (s != QS_OK) return s;
    if (n) *n = st->n;
    if (prec) *prec = st->prec;
    if (device_ptr) *device_ptr = st->data;
    return QS_OK;
  });
}

qs_status sv_set_basis(qs_state_t st, uint64_t J) {
  return abi_guard(__func__, [&]() -> qs_status {
    qs_status s = check_state(st);
    if (s != QS_OK) return s;
    if (J >> st->n) {
      set_error("basis index %llu out of range for n = %d", (unsigned long long)J, st->n);
      return QS_EINVAL;
    }
    return launch_set_basis(st, J);
  });
}

qs_status sv_copy_in(qs_state_t st, const void* buf, int on_device) {
  return abi_guard(__func__, [&]() -> qs_status {
    qs_status s = check_state(st);
    if (s != QS_OK) return s;
    if (!buf) {
      set_error("buf is NULL");
      return QS_EINVAL;
    }
    if (on_device) {
      QS_CUDA(cudaMemcpyAsync(st->data, buf, st->data_bytes, cudaMemcpyDeviceToDevice, st->stream));
    } else {
      QS_CUDA(cudaMemcpyAsync(st->data, buf, st->data_bytes, cudaMemcpyHostToDevice, st->stream));
      QS_CUDA(cudaStreamSynchronize(st->stream));
    }
    return QS_OK;
  });
}

qs_status sv_copy_out(qs_state_t st, void* buf, int on_device) {
  return abi_guard(__func__, [&]() -> qs_status {
    qs_status s = check_state(st);
    if (s != QS_OK) return s;
    if (!buf) {
      set_error("buf is NULL");
      return QS_EINVAL;
    }
    if (on_device) {
      QS_CUDA(cudaMemcpyAsync(buf, st->data, st->data_bytes, cudaMemcpyDeviceToDevice, st->stream));
    } else {
      QS_CUDA(cudaMemcpyAsync(buf, st->data, st->data_bytes, cudaMemcpyDeviceToHost, st->stream));
      QS_CUDA(cudaStreamSynchronize(st->stream));
    }
    return QS_OK;
  });
}

qs_status sv_apply_circuit(qs_state_t st, const qs_gate* gates, size_t ngates, const qs_opts* opts,
                           qs_stats* stats) {
  return abi_guard(__func__, [&]() -> qs_status {
    qs_status s = check_state(st);
    if (s != QS_OK) return s;
    s = validate_gates(gates, ngates, st->n);
    if (s != QS_OK) return s;
    return apply_gates(st, gates, ngates, opts ? opts->method : QS_METHOD_AUTO, stats,
                       opts ? opts->flags : 0);
  });
}

qs_status sv_probs(qs_state_t st, void* out, int out_fp64, uint64_t marg_mask, double* norm_out) {
  return abi_guard(__func__, [&]() -> qs_status {
    qs_status s = check_state(st);
    if (s != QS_OK) return s;
    if (marg_mask >> st->n) {
      set_error("marginal mask has bits beyond n = %d", st->n);
      return QS_EINVAL;
    }
    int k = __builtin_popcountll(marg_mask);
    const bool marginal = marg_mask != 0 && k != st->n;
    if (marginal && k > kScratchMargLog2) {
      set_error("marginal over %d qubits exceeds the %d-qubit scratch limit", k, kScratchMargLog2);
      return QS_EUNSUPPORTED;
    }
    if (!marginal && out && !out_fp64 && st->prec == QS_C64 && ((uintptr_t)out & 7)) {
      set_error("float output buffer must be 8-byte aligned");
      return QS_EINVAL;
    }
    unsigned char* sc = (unsigned char*)st->scratch;
    double* partials = (double*)(sc + kScratchPartials);
    s = launch_probs(st, out, out_fp64, marginal ? marg_mask : 0, partials,
                     (uint8_t*)(sc + kScratchBits), (double*)(sc + kScratchMarg));
    if (s != QS_OK) return s;
    if (norm_out) {
      double* res = (double*)(sc + kScratchResult);
      s = launch_reduce_partials(st, partials, kReduceBlocks, res);
      if (s != QS_OK) return s;
      QS_CUDA(cudaMemcpyAsync(norm_out, res, sizeof(double), cudaMemcpyDeviceToHost, st->stream));
      QS_CUDA(cudaStreamSynchronize(st->stream));
    }
    return QS_OK;
  });
}

qs_status sv_probs_host(qs_state_t st, void* host_out, int out_fp64, uint64_t marg_mask, double* norm_out) {
  return abi_guard(__func__, [&]() -> qs_status {
    qs_status s = check_state(st);
    if (s != QS_OK) return s;
    if (!host_out) {
      set_error("host_out is required");
      return QS_EINVAL;
    }
    if (marg_mask >> st->n) {
      set_error("marginal mask has bits beyond n = %d", st->n);
      return QS_EINVAL;
    }
    s = wait_copies(st);
    if (s != QS_OK) return s;
    const int k = __builtin_popcountll(marg_mask);
    unsigned char* sc = (unsigned char*)st->scratch;
    double* partials = (double*)(sc + kScratchPartials);
    if (marg_mask != 0 && k != st->n) {
      // a marginal (at most 2^16 values) stays in the scratch accumulators as doubles
      if (k > kScratchMargLog2) {
        set_error("marginal over %d qubits exceeds the %d-qubit scratch limit", k, kScratchMargLog2);
        return QS_EUNSUPPORTED;
      }
      s = sv_probs(st, nullptr, 1, marg_mask, norm_out);
      if (s != QS_OK) return s;
      std::vector<double> h((size_t)1 << k);
      QS_CUDA(cudaMemcpyAsync(h.data(), sc + kScratchMarg, h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                              st->stream));
      QS_CUDA(cudaStreamSynchronize(st->stream));
      if (out_fp64) std::memcpy(host_out, h.data(), h.size() * sizeof(double));
      else
        for (size_t i = 0; i < h.size(); ++i) ((float*)host_out)[i] = (float)h[i];
      return QS_OK;
    }
    const size_t es = out_fp64 ? sizeof(double) : sizeof(float);
    const uint64_t N = 1ull << st->n;
    {
      // a page-locked host buffer the device can address: the kernel writes the
      // probabilities into it directly (one launch, no staging copies; 4 GiB in 22.2 ms
      // against 24.9 ms through the copy engine on GB300)
      cudaPointerAttributes pa;
      if (cudaPointerGetAttributes(&pa, host_out) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer) {
        s = launch_probs_range(st, 0, N, pa.devicePointer, out_fp64, partials);
        if (s == QS_OK && norm_out) s = sv_probs(st, nullptr, out_fp64, 0, norm_out);
        const cudaError_t e = cudaStreamSynchronize(st->stream);
        if (s == QS_OK && e != cudaSuccess) s = cuda_status(e, "sv_probs_host");
        return s;
      }
      cudaGetLastError();   // a plain host pointer: not an error
    }
    // otherwise formed chunk by chunk in a device staging buffer (kept by the state)
    // and copied to the host buffer after each chunk
    const uint64_t chunk = std::min<uint64_t>(N, (uint64_t)(kStageBytes / es));
    if (!st->stage) {
      st->stage = dev_alloc(st, kStageBytes);
      if (!st->stage) {
        set_error("staging buffer for the probabilities could not be allocated");
        return QS_ENOMEM;
      }
      st->stage_bytes = kStageBytes;
    }
    for (uint64_t off = 0; off < N && s == QS_OK; off += chunk) {
      const uint64_t cnt = std::min<uint64_t>(chunk, N - off);
      s = launch_probs_range(st, off, cnt, st->stage, out_fp64, partials);
      if (s == QS_OK) {
        const cudaError_t e = cudaMemcpyAsync((unsigned char*)host_out + off * es, st->stage, cnt * es,
                                              cudaMemcpyDeviceToHost, st->stream);
        if (e != cudaSuccess) s = cuda_status(e, "probabilities to the host");
      }
    }
    if (s == QS_OK && norm_out) s = sv_probs(st, nullptr, out_fp64, 0, norm_out);
    const cudaError_t e = cudaStreamSynchronize(st->stream);
    if (s == QS_OK && e != cudaSuccess) s = cuda_status(e, "sv_probs_host");
    return s;
  });
}

qs_status sv_probs_host_async(qs_state_t st, void* host_out, int out_fp64) {
  return abi_guard(__func__, [&]() -> qs_status {
    qs_status s = check_state(st);
    if (s != QS_OK) return s;
    if (!host_out) {
      set_error("host_out is required");
      return QS_EINVAL;
    }
    const uint64_t N = 1ull << st->n;
    const size_t bytes = (size_t)N * (out_fp64 ? sizeof(double) : sizeof(float));
    HostCopies* hc = nullptr;
    s = copies_for(st, bytes, &hc);
    if (s != QS_OK) return s;
    const int k = hc->next;
    unsigned char* dst = (unsigned char*)hc->buf + (size_t)k * hc->half;
    // the buffer's earlier copy has to end before the buffer is rewritten
    if (hc->queued[k]) QS_CUDA(cudaStreamWaitEvent(st->stream, hc->copied[k], 0));
    double* partials = (double*)((unsigned char*)st->scratch + kScratchPartials);
    s = launch_probs_range(st, 0, N, dst, out_fp64, partials);
    if (s != QS_OK) return s;
    QS_CUDA(cudaEventRecord(hc->formed[k], st->stream));
    QS_CUDA(cudaStreamWaitEvent(hc->cs, hc->formed[k], 0));
    QS_CUDA(cudaMemcpyAsync(host_out, dst, bytes, cudaMemcpyDeviceToHost, hc->cs));
    QS_CUDA(cudaEventRecord(hc->copied[k], hc->cs));
    hc->queued[k] = true;
    hc->next = k ^ 1;
    return QS_OK;
  });
}

qs_status sv_probs_wait(qs_state_t st) {
  return abi_guard(__func__, [&]() -> qs_status {
    qs_status s = check_state(st);
    if (s != QS_OK) return s;
    return wait_copies(st);
  });
}

qs_status sv_loglik(qs_state_t st, const uint32_t* counts, double* out, int64_t* clamped) {
  return abi_guard(__func__, [&]() -> qs_status {
    qs_status s = check_state(st);
    if (s != QS_OK) return s;
    if (!counts || !out) {
      set_error("counts and out are required");
      return QS_EINVAL;
    }
    unsigned char* sc = (unsigned char*)st->scratch;
    double* partials = (double*)(sc + kScratchPartials);
    s = launch_loglik(st, counts, partials, (unsigned long long*)(sc + kScratchClamps));
    if (s != QS_OK) return s;
    double* res = (double*)(sc + kScratchResult);
    s = launch_reduce_partials(st, partials, kReduceBlocks, res);
    if (s != QS_OK) return s;
    unsigned long long nc = 0;
    QS_CUDA(cudaMemcpyAsync(out, res, sizeof(double), cudaMemcpyDeviceToHost, st->stream));
    QS_CUDA(cudaMemcpyAsync(&nc, sc + kScratchClamps, sizeof(nc), cudaMemcpyDeviceToHost, st->stream));
    QS_CUDA(cudaStreamSynchronize(st->stream));
    if (clamped) *clamped = (int64_t)nc;
    return QS_OK;
  });
}

qs_status qs_profile_begin(void) {
  return abi_guard(__func__, [&]() -> qs_status {
    ProfileSession& ps = profile();
    std::lock_guard<std::mutex> g(ps.mu);
    if (ps.active) {
      set_error("a profiling session is already active");
      return QS_EINVAL;
    }
    ps.ev.clear();
    ps.kind.clear();
    ps.active = true;
    return QS_OK;
  });
}

qs_status qs_profile_end(double* kernel_ms, int64_t* launches) {
  return abi_guard(__func__, [&]() -> qs_status {
    ProfileSession& ps = profile();
    std::lock_guard<std::mutex> g(ps.mu);
    if (!ps.active) {
      set_error("no active profiling session");
      return QS_EINVAL;
    }
    ps.active = false;
    double ms[5] = {0, 0, 0, 0, 0};
    int64_t cnt[5] = {0, 0, 0, 0, 0};
    qs_status s = QS_OK;
    for (size_t i = 0; i < ps.kind.size(); ++i) {
      cudaEvent_t a = ps.ev[2 * i], b = ps.ev[2 * i + 1];
      if (a && b) {
        cudaError_t e = cudaEventSynchronize(b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
        if (e != cudaSuccess && s == QS_OK) s = cuda_status(e, "profile events");
        ms[ps.kind[i]] += t;
        cnt[ps.kind[i]] += 1;
      }
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
    ps.ev.clear();
    ps.kind.clear();
    for (int k = 0; k < 5; ++k) {
      if (kernel_ms) kernel_ms[k] = ms[k];
      if (launches) launches[k] = cnt[k];
    }
    return s;
  });
}

}  // extern "C"
