// Serving loop: continuous batching of state-vector circuits on one GPU.
//
// A scheduler thread owns every CUDA call of a server.  Circuits arrive
// through qs_server_submit at any time; each scheduler iteration
//   1. retires finished work (CUDA events), records latencies, frees states;
//   2. admits waiting circuits while slots and device memory allow:
//      - small circuits (n <= small_max_qubits) go into the next packed launch,
//        one CTA per circuit with the whole state in shared memory, started as
//        soon as the previous packed launch has finished;
//      - larger circuits get a resident state allocated stream-ordered on one
//        of max_inflight streams, within mem_budget, and run the tiled pass
//        pipeline there, overlapping with the other streams;
//   3. sleeps briefly when nothing changed.
// The result of a circuit is the marginal outcome distribution over its mask
// (Born rule), copied to pinned host memory before its completion event.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "dev_common.cuh"
#include "internal.h"

namespace qs {
namespace {

constexpr int kMaxMargBits = 12;

struct SmallJob {
  int32_t n, k;
  int32_t op_begin, op_count;
  int64_t out_off;
  uint8_t bits[16];   // marginal bit positions
};

// One CTA per small circuit: |0...0>, all its ops in shared memory, marginal
// probabilities (fp64 accumulation) written to out.
template <typename R>
__global__ void __launch_bounds__(256)
    packed_small_kernel(const SmallJob* __restrict__ jobs, const PlainOp<R>* __restrict__ ops,
                        double* __restrict__ out, int max_n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<R>* sm = reinterpret_cast<C2<R>*>(smem_raw);
  double* hist = reinterpret_cast<double*>(smem_raw + (sizeof(C2<R>) << max_n));
  const SmallJob job = jobs[blockIdx.x];
  const int N = 1 << job.n, H = 1 << job.k;
  for (int J = threadIdx.x; J < N; J += blockDim.x) {
    C2<R> z;
    z.x = R(J == 0 ? 1 : 0);
    z.y = R(0);
    sm[J] = z;
  }
  for (int i = threadIdx.x; i < H; i += blockDim.x) hist[i] = 0.0;
  __syncthreads();
  small_apply_ops(sm, job.n, ops + job.op_begin, job.op_count);
  for (int J = threadIdx.x; J < N; J += blockDim.x) {
    const C2<R> a = sm[J];
    int K = 0;
    for (int i = 0; i < job.k; ++i) K |= ((J >> job.bits[i]) & 1) << i;
    atomicAdd(hist + K, (double)a.x * (double)a.x + (double)a.y * (double)a.y);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < H; i += blockDim.x) out[job.out_off + i] = hist[i];
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Req {
  int64_t id = 0;
  int n = 0, k = 0;
  uint64_t mask = 0;
  std::vector<qs_gate> gates;
  double t_submit = 0, t_done = 0;
  bool done = false;
  qs_status status = QS_OK;
  std::string err;
  std::vector<double> result;
  // large circuits in flight
  qs_state_t st = nullptr;
  int slot = -1;
  size_t bytes = 0;
};

// stream-ordered allocator for resident states
void* async_alloc(size_t bytes, void* stream, void*) {
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void async_free(void* p, size_t, void* stream, void*) { cudaFreeAsync(p, (cudaStream_t)stream); }

}  // namespace

struct Server {
  qs_server_config cfg{};
  int device = 0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::deque<Req*> pending;
  std::unordered_map<int64_t, Req*> reqs;
  int64_t next_id = 1;
  // large circuits
  std::vector<cudaStream_t> streams;
  std::vector<Req*> slot_req;
  std::vector<cudaEvent_t> slot_ev;
  std::vector<double*> slot_host;   // pinned results
  uint64_t bytes_in_use = 0, peak_bytes = 0;
  // packed launches
  cudaStream_t small_stream = nullptr;
  cudaEvent_t batch_ev = nullptr;
  std::vector<Req*> batch;
  bool batch_busy = false;
  void* d_buf = nullptr;
  size_t d_buf_bytes = 0;
  unsigned char* h_buf = nullptr;   // pinned: descriptors up, results down
  size_t h_buf_bytes = 0;
  size_t batch_out_off = 0;
  // statistics
  std::vector<double> lat_ms;
  double t_first = -1, t_last = 0;
  int64_t submitted = 0, completed = 0, packed_launches = 0, packed_circuits = 0, large_circuits = 0;

  void finish(Req* r, qs_status s) {
    r->status = s;
    if (s != QS_OK) r->err = qs_last_error();
    r->t_done = now_s();
    std::lock_guard<std::mutex> g(mu);
    r->done = true;
    lat_ms.push_back(1e3 * (r->t_done - r->t_submit));
    t_last = std::max(t_last, r->t_done);
    ++completed;
    cv_done.notify_all();
  }

  qs_status grow_buffers(size_t dev_bytes, size_t host_bytes) {
    if (dev_bytes > d_buf_bytes) {
      if (d_buf) cudaFree(d_buf);
      size_t want = std::max(dev_bytes, 2 * d_buf_bytes);
      if (cudaMalloc(&d_buf, want) != cudaSuccess) {
        cudaGetLastError();
        d_buf = nullptr;
        d_buf_bytes = 0;
        set_error("packed-launch buffer allocation failed");
        return QS_ENOMEM;
      }
      d_buf_bytes = want;
    }
    if (host_bytes > h_buf_bytes) {
      if (h_buf) cudaFreeHost(h_buf);
      size_t want = std::max(host_bytes, 2 * h_buf_bytes);
      if (cudaMallocHost((void**)&h_buf, want) != cudaSuccess) {
        cudaGetLastError();
        h_buf = nullptr;
        h_buf_bytes = 0;
        set_error("pinned buffer allocation failed");
        return QS_ENOMEM;
      }
      h_buf_bytes = want;
    }
    return QS_OK;
  }

  template <typename R>
  qs_status start_batch_t(std::vector<Req*>& jobs_in) {
    std::vector<SmallJob> jobs;
    std::vector<PlainOp<R>> ops;
    int max_n = 1, max_k = 0;
    int64_t out = 0;
    auto c2 = [](cd z) {
      C2<R> v;
      v.x = (R)z.real();
      v.y = (R)z.imag();
      return v;
    };
    for (Req* r : jobs_in) {
      std::vector<FOp> fops;
      std::vector<int> vmap;
      build_fused_ops(r->gates.data(), r->gates.size(), r->n, fops, vmap, true, false);
      SmallJob j{};
      j.n = r->n;
      j.k = r->k;
      j.op_begin = (int32_t)ops.size();
      j.op_count = (int32_t)fops.size();
      j.out_off = out;
      int kk = 0;
      for (int b = 0; b < r->n; ++b)
        if ((r->mask >> b) & 1) j.bits[kk++] = (uint8_t)b;
      jobs.push_back(j);
      out += (int64_t)1 << r->k;
      for (const FOp& o : fops) {
        PlainOp<R> p;
        std::memset(&p, 0, sizeof(p));
        p.type = o.type;
        p.t = o.t;
        p.c = o.c;
        p.a = o.a;
        p.b = o.b;
        if (o.type == F_G1) {
          for (int i = 0; i < 4; ++i) p.m[i] = c2(o.m0[i]);
        } else if (o.type == F_G1C) {
          for (int i = 0; i < 4; ++i) p.m[i] = c2(o.m0[i]), p.m[4 + i] = c2(o.m1[i]);
        } else if (o.type == F_D) {
          for (int i = 0; i < 4; ++i) p.m[i] = c2(o.d[i]);
        } else {
          for (int i = 0; i < 16; ++i) p.m[i] = c2(o.g[i]);
        }
        ops.push_back(p);
      }
      max_n = std::max(max_n, r->n);
      max_k = std::max(max_k, r->k);
    }
    const size_t jb = (sizeof(SmallJob) * jobs.size() + 255) & ~size_t(255);
    const size_t ob = (sizeof(PlainOp<R>) * ops.size() + 255) & ~size_t(255);
    const size_t rb = sizeof(double) * (size_t)out;
    qs_status s = grow_buffers(jb + ob + rb, std::max(jb + ob, rb));
    if (s != QS_OK) return s;
    std::memcpy(h_buf, jobs.data(), sizeof(SmallJob) * jobs.size());
    if (!ops.empty()) std::memcpy(h_buf + jb, ops.data(), sizeof(PlainOp<R>) * ops.size());
    unsigned char* d = (unsigned char*)d_buf;
    QS_CUDA(cudaMemcpyAsync(d, h_buf, jb + ob, cudaMemcpyHostToDevice, small_stream));
    const size_t smem = (sizeof(C2<R>) << max_n) + (sizeof(double) << max_k);
    if (smem > 48 * 1024)
      QS_CUDA(cudaFuncSetAttribute(packed_small_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    packed_small_kernel<R><<<(unsigned)jobs.size(), 256, smem, small_stream>>>(
        (const SmallJob*)d, (const PlainOp<R>*)(d + jb), (double*)(d + jb + ob), max_n);
    QS_CUDA(cudaGetLastError());
    QS_CUDA(cudaMemcpyAsync(h_buf, d + jb + ob, rb, cudaMemcpyDeviceToHost, small_stream));
    QS_CUDA(cudaEventRecord(batch_ev, small_stream));
    batch = jobs_in;
    batch_busy = true;
    ++packed_launches;
    packed_circuits += (int64_t)jobs_in.size();
    return QS_OK;
  }

  void start_batch(std::vector<Req*>& jobs) {
    qs_status s = cfg.prec == QS_C64 ? start_batch_t<float>(jobs) : start_batch_t<double>(jobs);
    if (s != QS_OK) {
      cudaStreamSynchronize(small_stream);
      for (Req* r : jobs) finish(r, s);
      batch.clear();
      batch_busy = false;
    }
  }

  void finish_batch() {
    size_t off = 0;
    for (Req* r : batch) {
      const size_t H = (size_t)1 << r->k;
      r->result.assign((double*)h_buf + off, (double*)h_buf + off + H);
      off += H;
      finish(r, QS_OK);
    }
    batch.clear();
    batch_busy = false;
  }

  void start_large(Req* r, int slot) {
    qs_allocator a{async_alloc, async_free, nullptr};
    qs_status s = sv_create(r->n, cfg.prec, &a, streams[slot], &r->st);
    if (s == QS_OK) s = apply_gates(r->st, r->gates.data(), r->gates.size(), QS_METHOD_TILED, nullptr);
    if (s == QS_OK) {
      unsigned char* sc = (unsigned char*)r->st->scratch;
      double* marg = (double*)(sc + kScratchMarg);
      // a mask covering all n bits is the plain distribution (written to the same place)
      const bool all = r->k == r->n;
      s = launch_probs(r->st, all ? marg : nullptr, 1, all ? 0 : r->mask,
                       (double*)(sc + kScratchPartials), (uint8_t*)(sc + kScratchBits), marg);
      if (s == QS_OK) {
        cudaError_t e = cudaMemcpyAsync(slot_host[slot], sc + kScratchMarg, sizeof(double) << r->k,
                                        cudaMemcpyDeviceToHost, streams[slot]);
        if (e == cudaSuccess) e = cudaEventRecord(slot_ev[slot], streams[slot]);
        if (e != cudaSuccess) s = cuda_status(e, "large circuit readout");
      }
    }
    r->slot = slot;
    slot_req[slot] = r;
    ++large_circuits;
    if (s != QS_OK) {
      cudaStreamSynchronize(streams[slot]);
      release_large(r);
      finish(r, s);
    }
  }

  void release_large(Req* r) {
    if (r->st) sv_destroy(r->st);
    r->st = nullptr;
    if (r->slot >= 0) slot_req[r->slot] = nullptr;
    {
      std::lock_guard<std::mutex> g(mu);
      bytes_in_use -= r->bytes;
    }
    r->slot = -1;
  }

  void finish_large(Req* r) {
    const int slot = r->slot;
    r->result.assign(slot_host[slot], slot_host[slot] + ((size_t)1 << r->k));
    release_large(r);
    finish(r, QS_OK);
  }

  // Event query with a testing hook: qs_server_inject_query_error makes the next
  // query return a given error instead of asking the device.
  std::atomic<int> injected_error{0};
  cudaError_t query(cudaEvent_t ev) {
    const int inj = injected_error.exchange(0);
    if (inj != 0) return (cudaError_t)inj;
    return cudaEventQuery(ev);
  }

  void fail_large(Req* r, cudaError_t e) {
    cudaGetLastError();   // clears a non-sticky error
    const qs_status st = cuda_status(e, "completion of a large circuit");
    const std::string msg = qs_last_error();
    cudaStreamSynchronize(streams[r->slot]);   // nothing of it may still write its buffers
    cudaGetLastError();
    release_large(r);
    set_error("%s", msg.c_str());
    finish(r, st);
  }

  void fail_batch(cudaError_t e) {
    cudaGetLastError();
    const qs_status st = cuda_status(e, "completion of a packed launch");
    const std::string msg = qs_last_error();
    cudaStreamSynchronize(small_stream);
    cudaGetLastError();
    for (Req* r : batch) {
      set_error("%s", msg.c_str());
      finish(r, st);
    }
    batch.clear();
    batch_busy = false;
  }

  void run() {
    cudaSetDevice(device);
    for (;;) {
      bool progress = false;
      // 1. retire finished work; a query that reports an error (neither done nor
      // still running) completes the work with that error
      for (size_t s = 0; s < slot_req.size(); ++s) {
        Req* r = slot_req[s];
        if (!r) continue;
        const cudaError_t e = query(slot_ev[s]);
        if (e == cudaSuccess) {
          finish_large(r);
          progress = true;
        } else if (e != cudaErrorNotReady) {
          fail_large(r, e);
          progress = true;
        }
      }
      if (batch_busy) {
        const cudaError_t e = query(batch_ev);
        if (e == cudaSuccess) {
          finish_batch();
          progress = true;
        } else if (e != cudaErrorNotReady) {
          fail_batch(e);
          progress = true;
        }
      }
      // 2. admission
      std::vector<Req*> to_batch, too_big;
      std::vector<std::pair<Req*, int>> to_large;
      {
        std::lock_guard<std::mutex> g(mu);
        bool idle = pending.empty() && !batch_busy &&
                    std::all_of(slot_req.begin(), slot_req.end(), [](Req* x) { return x == nullptr; });
        if (stop && idle) return;
        std::vector<bool> busy(slot_req.size());
        for (size_t s = 0; s < slot_req.size(); ++s) busy[s] = slot_req[s] != nullptr;
        for (auto it = pending.begin(); it != pending.end();) {
          Req* r = *it;
          if (r->n <= cfg.small_max_qubits) {
            if (!batch_busy && (int)to_batch.size() < cfg.max_batch) {
              to_batch.push_back(r);
              it = pending.erase(it);
              continue;
            }
          } else {
            int slot = -1;
            for (size_t s = 0; s < busy.size(); ++s)
              if (!busy[s]) {
                slot = (int)s;
                break;
              }
            const size_t need = ((size_t)(cfg.prec == QS_C64 ? 8 : 16) << r->n) + kScratchBytes + (4u << 20);
            if (need > cfg.mem_budget) {   // can never be admitted
              too_big.push_back(r);
              it = pending.erase(it);
              continue;
            }
            if (slot >= 0 && bytes_in_use + need <= cfg.mem_budget) {
              busy[slot] = true;
              r->bytes = need;
              bytes_in_use += need;
              peak_bytes = std::max(peak_bytes, bytes_in_use);
              to_large.push_back({r, slot});
              it = pending.erase(it);
              continue;
            }
          }
          ++it;
        }
      }
      for (Req* r : too_big) {
        set_error("circuit of %d qubits needs more device memory than the server budget", r->n);
        finish(r, QS_ENOMEM);
        progress = true;
      }
      if (!to_batch.empty()) {
        start_batch(to_batch);
        progress = true;
      }
      for (auto& p : to_large) {
        start_large(p.first, p.second);
        progress = true;
      }
      if (!progress) {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait_for(lk, std::chrono::microseconds(20));
      }
    }
  }
};

}  // namespace qs

using namespace qs;

struct qs_server_s : public qs::Server {};

extern "C" {

qs_status qs_server_create(const qs_server_config* cfg, qs_server_t* out) {
  if (!cfg || !out) {
    set_error("cfg and out are required");
    return QS_EINVAL;
  }
  *out = nullptr;
  if (cfg->prec != QS_C64 && cfg->prec != QS_C128) {
    set_error("bad precision");
    return QS_EINVAL;
  }
  const int small_cap = cfg->prec == QS_C64 ? 14 : 13;
  if (cfg->small_max_qubits < 0 || cfg->small_max_qubits > small_cap || cfg->max_inflight < 0 ||
      cfg->max_batch < 0) {
    set_error("bad server configuration");
    return QS_EINVAL;
  }
  qs_server_s* s = new (std::nothrow) qs_server_s();
  if (!s) return QS_ENOMEM;
  s->cfg = *cfg;
  if (s->cfg.small_max_qubits == 0) s->cfg.small_max_qubits = small_cap;
  if (s->cfg.max_inflight == 0) s->cfg.max_inflight = 4;
  if (s->cfg.max_batch == 0) s->cfg.max_batch = 1024;
  cudaGetDevice(&s->device);
  if (s->cfg.mem_budget == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    s->cfg.mem_budget = (uint64_t)(0.8 * (double)fr);
  }
  const int m = s->cfg.max_inflight;
  s->streams.resize(m);
  s->slot_req.assign(m, nullptr);
  s->slot_ev.resize(m);
  s->slot_host.resize(m);
  for (int i = 0; i < m; ++i) {
    cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&s->slot_ev[i], cudaEventDisableTiming);
    cudaMallocHost((void**)&s->slot_host[i], sizeof(double) << kMaxMargBits);
  }
  cudaStreamCreateWithFlags(&s->small_stream, cudaStreamNonBlocking);
  cudaEventCreateWithFlags(&s->batch_ev, cudaEventDisableTiming);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    qs_status st = cuda_status(e, "server setup");
    delete s;
    return st;
  }
  s->worker = std::thread([s]() { s->run(); });
  *out = s;
  return QS_OK;
}

qs_status qs_server_submit(qs_server_t s, int n, const qs_gate* gates, size_t ngates,
                           uint64_t marg_mask, int64_t* ticket) {
  if (!s || !ticket) {
    set_error("server and ticket are required");
    return QS_EINVAL;
  }
  if (n < 1 || n > 30) {
    set_error("n = %d outside [1, 30]", n);
    return QS_EINVAL;
  }
  if (marg_mask >> n) {
    set_error("mask has bits beyond n");
    return QS_EINVAL;
  }
  uint64_t mask = marg_mask ? marg_mask : (n <= kMaxMargBits ? ((1ull << n) - 1) : 0);
  const int k = __builtin_popcountll(mask);
  if (k == 0 || k > kMaxMargBits) {
    set_error("marginal over %d qubits: must be 1..%d", k, kMaxMargBits);
    return QS_EINVAL;
  }
  qs_status st = validate_gates(gates, ngates, n);
  if (st != QS_OK) return st;
  Req* r = new (std::nothrow) Req();
  if (!r) return QS_ENOMEM;
  r->n = n;
  r->mask = mask;
  r->k = k;
  r->gates.assign(gates, gates + ngates);
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> g(s->mu);
    r->id = s->next_id++;
    s->reqs[r->id] = r;
    s->pending.push_back(r);
    ++s->submitted;
    if (s->t_first < 0) s->t_first = r->t_submit;
  }
  s->cv_work.notify_one();
  *ticket = r->id;
  return QS_OK;
}

qs_status qs_server_wait(qs_server_t s, int64_t ticket, double* result, double* latency_ms) {
  if (!s) {
    set_error("server is NULL");
    return QS_EINVAL;
  }
  Req* r = nullptr;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
      set_error("unknown ticket %lld", (long long)ticket);
      return QS_EINVAL;
    }
    r = it->second;
    s->cv_done.wait(lk, [r]() { return r->done; });
    s->reqs.erase(it);
  }
  qs_status st = r->status;
  if (st != QS_OK) set_error("%s", r->err.c_str());
  if (st == QS_OK && result) std::memcpy(result, r->result.data(), sizeof(double) * r->result.size());
  if (latency_ms) *latency_ms = 1e3 * (r->t_done - r->t_submit);
  delete r;
  return st;
}

qs_status qs_server_stats_get(qs_server_t s, qs_server_stats* out) {
  if (!s || !out) {
    set_error("server and out are required");
    return QS_EINVAL;
  }
  std::lock_guard<std::mutex> g(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->packed_launches = s->packed_launches;
  out->packed_circuits = s->packed_circuits;
  out->large_circuits = s->large_circuits;
  out->peak_bytes = s->peak_bytes;
  std::vector<double> l = s->lat_ms;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) {
      const double pos = q * (double)(l.size() - 1);
      const size_t i = (size_t)pos;
      const double f = pos - (double)i;
      return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double sum = 0;
    for (double x : l) sum += x;
    out->mean_ms = sum / (double)l.size();
    out->max_ms = l.back();
    out->wall_s = s->t_last - s->t_first;
    out->circuits_per_s = out->wall_s > 0 ? (double)s->completed / out->wall_s : 0.0;
  }
  return QS_OK;
}

qs_status qs_server_inject_query_error(qs_server_t s, int cuda_error) {
  if (!s || cuda_error <= 0 || cuda_error == (int)cudaErrorNotReady) {
    set_error("server and a CUDA error code other than cudaErrorNotReady are required");
    return QS_EINVAL;
  }
  s->injected_error.store(cuda_error);
  return QS_OK;
}

qs_status qs_server_destroy(qs_server_t s) {
  if (!s) return QS_OK;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->reqs) delete kv.second;
  for (size_t i = 0; i < s->streams.size(); ++i) {
    cudaStreamDestroy(s->streams[i]);
    cudaEventDestroy(s->slot_ev[i]);
    cudaFreeHost(s->slot_host[i]);
  }
  cudaStreamDestroy(s->small_stream);
  cudaEventDestroy(s->batch_ev);
  if (s->d_buf) cudaFree(s->d_buf);
  if (s->h_buf) cudaFreeHost(s->h_buf);
  delete s;
  return QS_OK;
}

}  // extern "C"
