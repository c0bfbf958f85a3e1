// Serving loop: continuous batching of state-vector circuits on one GPU.
//
// Small circuits (n <= small_max_qubits) go through one persistent packed
// kernel fed by a work queue that lives in page-locked, device-mapped host
// memory:
//   - the scheduler thread fuses a circuit's gates on the host, writes its ops
//     into an op arena and a job descriptor into a ring, and publishes the job by
//     advancing the ring's tail (a release store);
//   - each CTA of the persistent kernel claims the next published job with an
//     atomic on a device counter, stages its ops in shared memory, runs the
//     whole circuit on a state held in shared memory, reduces the marginal
//     outcome probabilities (Born rule, FP64 accumulation) into a result arena,
//     and sets the job's done word (a release store at system scope), which the
//     scheduler polls;
//   - a CTA that finds no published job waits at most idle_ms (a globaltimer
//     deadline), then ends and the kernel reports QS_ETIMEOUT in its status word;
//     the scheduler counts it and launches the kernel again when work arrives.
//     The kernel also ends after a maximum lifetime (50 ms), which offers its SMs
//     to tensor-core block passes waiting for whole SMs.
// While the persistent kernel may run it holds up to persistent_ctas SMs, and the
// block passes of the library leave that many SMs free.
//
// Larger circuits are admitted as device memory and worker slots free up: each of
// max_inflight worker threads owns a stream, creates a resident state (stream-
// ordered allocation within mem_budget), applies the gates with the default
// method (QS_METHOD_AUTO: dense blocks on the tensor cores, the rest in tile
// passes; QS_METHOD_TILED when configured) and reads back the marginal.  The
// packed kernel and the workers overlap on the device.
// Latency = completion seen by the scheduler (small) or the worker (large) -
// submission time.
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

#include "abi_guard.h"
#include "fuse_merge.h"
#include "dev_common.cuh"
#include "internal.h"

namespace qs {

// SMs the block passes leave free for running persistent packed kernels
std::atomic<int> g_reserved_sms{0};
int reserved_sms() { return g_reserved_sms.load(); }

namespace {

constexpr int kMaxMargBits = 12;
constexpr int kOpChunk = 32;             // ops staged in shared memory at a time
constexpr int64_t kRing = 4096;          // job ring entries
constexpr int64_t kOpArena = 1 << 19;    // ops in the op arena
constexpr int64_t kResArena = 1 << 22;   // doubles in the result arena
constexpr uint64_t kLifeNs = 50000000ull;

struct alignas(16) PJob {
  int32_t n, k, nops, pad;
  int64_t op_off;    // first op of the job in the op arena
  int64_t out_off;   // first double of its marginal in the result arena
  uint8_t bits[16];  // bit positions of the marginal
};

struct PCtl {        // written by the host, read by the kernel
  uint64_t tail;     // jobs published so far
  uint32_t stop;     // nonzero: CTAs end instead of waiting
  uint32_t pad[13];
};

__device__ __forceinline__ uint64_t ld_acquire_sys(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_sys(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(uint32_t* p, uint32_t v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <typename R>
__global__ void __launch_bounds__(256)
    packed_persistent_kernel(const PCtl* __restrict__ ctl, const PJob* __restrict__ jobs,
                             const PlainOp<R>* __restrict__ ops, double* __restrict__ results,
                             uint32_t* __restrict__ done, unsigned long long* __restrict__ head,
                             int* __restrict__ status, int max_n, uint64_t idle_ns, uint64_t life_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<R>* sm = reinterpret_cast<C2<R>*>(smem_raw);
  double* hist = reinterpret_cast<double*>(smem_raw + (sizeof(C2<R>) << max_n));
  PlainOp<R>* chunk = reinterpret_cast<PlainOp<R>*>(smem_raw + (sizeof(C2<R>) << max_n) +
                                                    (sizeof(double) << kMaxMargBits));
  __shared__ long long s_job;
  __shared__ PJob s_desc;
  const uint64_t born = gtimer();
  for (;;) {
    if (threadIdx.x == 0) {
      // claim the next published job; wait for one at most idle_ns
      long long got = -1;
      const uint64_t t0 = gtimer();
      for (;;) {
        const unsigned long long h = atomicAdd(head, 0ull);
        const uint64_t tail = ld_acquire_sys(&ctl->tail);
        if (h < tail) {
          if (atomicCAS(head, h, h + 1ull) == h) {
            got = (long long)h;
            break;
          }
          continue;
        }
        const uint64_t now = gtimer();
        if (ld_relaxed_sys(&ctl->stop) != 0u || now - born > life_ns) break;
        if (now - t0 > idle_ns) {   // no producer within the limit
          atomicMax(status, (int)QS_ETIMEOUT);
          break;
        }
        __nanosleep(256);
      }
      s_job = got;
      if (got >= 0) {   // written before the tail it was published with; read past the caches
        const uint4* src = reinterpret_cast<const uint4*>(jobs + got % kRing);
        uint4* dst = reinterpret_cast<uint4*>(&s_desc);
        for (int w = 0; w < (int)(sizeof(PJob) / 16); ++w) dst[w] = __ldcv(src + w);
      }
    }
    __syncthreads();
    const long long j = s_job;
    if (j < 0) return;
    const PJob job = s_desc;
    const int N = 1 << job.n, H = 1 << job.k;
    for (int J = threadIdx.x; J < N; J += blockDim.x) {
      C2<R> z;
      z.x = R(J == 0 ? 1 : 0);
      z.y = R(0);
      sm[J] = z;
    }
    for (int i = threadIdx.x; i < H; i += blockDim.x) hist[i] = 0.0;
    // the ops in chunks: a coalesced copy into shared memory, then applied in order
    for (int o0 = 0; o0 < job.nops; o0 += kOpChunk) {
      const int cnt = min(kOpChunk, job.nops - o0);
      const uint4* src = reinterpret_cast<const uint4*>(ops + job.op_off + o0);
      uint4* dst = reinterpret_cast<uint4*>(chunk);
      const int words = cnt * (int)(sizeof(PlainOp<R>) / 16);
      __syncthreads();   // nobody reads the previous chunk any more
      for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = __ldcv(src + w);
      __syncthreads();
      small_apply_ops(sm, job.n, chunk, cnt);
    }
    __syncthreads();
    for (int J = threadIdx.x; J < N; J += blockDim.x) {
      const C2<R> a = sm[J];
      int K = 0;
      for (int i = 0; i < job.k; ++i) K |= ((J >> job.bits[i]) & 1) << i;
      atomicAdd(hist + K, (double)a.x * (double)a.x + (double)a.y * (double)a.y);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < H; i += blockDim.x) results[job.out_off + i] = hist[i];
    __threadfence_system();
    __syncthreads();
    if (threadIdx.x == 0) st_release_sys(done + (j % kRing), (uint32_t)(j + 1));
  }
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
  size_t bytes = 0;          // large circuits: admitted device bytes
};

// a published small job (the scheduler's own record; its Req may be gone once
// the job is finished and waited for)
struct QJob {
  Req* r = nullptr;          // null once finished
  int64_t job = 0;
  int k = 0;
  int64_t out_off = 0;
  int64_t op_start = 0, res_start = 0;   // arena counters where its ranges began
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

// a contiguous range of `want` entries of a ring arena of `cap` entries with
// monotonic counters head (next free) and tail (oldest in use); a range never
// wraps (it starts over at entry 0 instead)
bool arena_take(int64_t& head, int64_t tail, int64_t cap, int64_t want, int64_t* at) {
  const int64_t pos = head % cap;
  const int64_t pad = pos + want > cap ? cap - pos : 0;
  if (want > cap || head + pad + want - tail > cap) return false;
  *at = (head + pad) % cap;
  head += pad + want;
  return true;
}

}  // namespace

struct Server {
  qs_server_config cfg{};
  int device = 0, sms = 152;
  std::thread scheduler;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_large;
  bool stop = false, stop_workers = false;
  std::deque<Req*> pending;          // submitted, not yet admitted
  std::deque<Req*> large_queue;      // admitted large circuits waiting for a worker
  std::unordered_map<int64_t, Req*> reqs;
  int64_t next_id = 1;
  uint64_t bytes_in_use = 0, peak_bytes = 0;
  int large_running = 0;
  // persistent packed kernel and its queue
  cudaStream_t pk_stream = nullptr;
  cudaEvent_t pk_ev = nullptr;
  bool pk_running = false;
  int pk_reserved = 0;
  size_t pk_smem = 0, op_size = 0;
  PCtl* ctl = nullptr;               // mapped host memory from here ...
  PJob* jobs = nullptr;
  uint32_t* done_words = nullptr;
  unsigned char* op_arena = nullptr;
  double* res_arena = nullptr;       // ... to here
  unsigned long long* d_head = nullptr;
  int* d_status = nullptr;
  int64_t published = 0;
  std::deque<QJob> in_queue;         // published jobs in publish order, until retired from the front
  std::vector<FOp> fops_scratch;     // fused ops of the circuit being published
  std::vector<int> vmap_scratch;
  std::vector<int> merge_scratch;    // its merge marks
  int64_t op_head = 0, op_tail = 0, res_head = 0, res_tail = 0;
  // statistics
  std::vector<double> lat_ms;
  double t_first = -1, t_last = 0;
  int64_t submitted = 0, completed = 0, packed_launches = 0, packed_circuits = 0, large_circuits = 0,
          idle_timeouts = 0;
  std::atomic<int> injected_error{0};

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

  // ---------------------------------------------------------------- small circuits
  template <typename R>
  bool publish_t(Req* r) {
    const int64_t oldest = in_queue.empty() ? published : in_queue.front().job;
    if (published - oldest >= kRing) return false;   // ring full
    std::vector<FOp>& fops = fops_scratch;   // the scheduler thread's, reused across circuits
    build_fused_ops(r->gates.data(), r->gates.size(), r->n, fops, vmap_scratch, true, false);
    // one CTA runs the whole circuit: one-qubit ops merged over the whole list
    // (marked in place; the merged ones are skipped below)
    std::vector<int>& into = merge_scratch;
    mark_one_qubit_merges(fops, r->n, &into);
    int64_t nops = 0;
    for (int v : into) nops += v < 0 ? 1 : 0;
    const int64_t H = (int64_t)1 << r->k;
    int64_t oh = op_head, rh = res_head, op_at = 0, res_at = 0;
    if (!arena_take(oh, op_tail, kOpArena, nops, &op_at) || !arena_take(rh, res_tail, kResArena, H, &res_at))
      return false;   // wait for finished jobs to free arena space
    auto c2 = [](cd z) {
      C2<R> v;
      v.x = (R)z.real();
      v.y = (R)z.imag();
      return v;
    };
    PlainOp<R>* dst = reinterpret_cast<PlainOp<R>*>(op_arena) + op_at;
    for (size_t i = 0, k = 0; i < fops.size(); ++i) {
      if (into[i] >= 0) continue;
      const FOp& o = fops[i];
      PlainOp<R> p;
      std::memset(&p, 0, sizeof(p));
      p.type = o.type;
      p.t = o.t;
      p.c = o.c;
      p.a = o.a;
      p.b = o.b;
      if (o.type == F_G1) {
        for (int q = 0; q < 4; ++q) p.m[q] = c2(o.m0[q]);
      } else if (o.type == F_G1C) {
        for (int q = 0; q < 4; ++q) p.m[q] = c2(o.m0[q]), p.m[4 + q] = c2(o.m1[q]);
      } else if (o.type == F_D) {
        for (int q = 0; q < 4; ++q) p.m[q] = c2(o.d[q]);
      } else {
        for (int q = 0; q < 16; ++q) p.m[q] = c2(o.g[q]);
      }
      dst[k++] = p;
    }
    QJob q;
    q.r = r;
    q.job = published;
    q.k = r->k;
    q.out_off = res_at;
    q.op_start = op_head;
    q.res_start = res_head;
    op_head = oh;
    res_head = rh;
    PJob& jd = jobs[published % kRing];
    jd.n = r->n;
    jd.k = r->k;
    jd.nops = (int32_t)nops;
    jd.pad = 0;
    jd.op_off = op_at;
    jd.out_off = res_at;
    std::memset(jd.bits, 0, sizeof(jd.bits));
    for (int b = 0, kk = 0; b < r->n; ++b)
      if ((r->mask >> b) & 1) jd.bits[kk++] = (uint8_t)b;
    // ops, descriptor and the cleared done word are written before the tail
    reinterpret_cast<std::atomic<uint32_t>*>(done_words + published % kRing)->store(0u, std::memory_order_relaxed);
    ++published;
    reinterpret_cast<std::atomic<uint64_t>*>(&ctl->tail)->store((uint64_t)published, std::memory_order_release);
    in_queue.push_back(q);
    ++packed_circuits;
    return true;
  }
  // true once r is taken (published, or failed: a host allocation in the fusion
  // failed before anything was written, and r's wait returns that error)
  bool publish(Req* r) {
    bool taken = false;
    const qs_status s = abi_guard("publishing a small circuit", [&]() -> qs_status {
      taken = cfg.prec == QS_C64 ? publish_t<float>(r) : publish_t<double>(r);
      return QS_OK;
    });
    if (s != QS_OK) {
      finish(r, s);
      return true;
    }
    return taken;
  }

  // finished jobs (done word set), in any order; arena space is reclaimed over
  // the finished prefix of the queue
  bool retire_small() {
    bool any = false;
    // jobs are claimed in publish order and at most persistent_ctas run at a time,
    // so only the first unfinished ones can have finished
    int unfinished_seen = 0;
    for (QJob& q : in_queue) {
      if (!q.r) continue;
      if (++unfinished_seen > 2 * cfg.persistent_ctas + 8) break;
      const uint32_t w =
          reinterpret_cast<std::atomic<uint32_t>*>(done_words + q.job % kRing)->load(std::memory_order_acquire);
      if (w != (uint32_t)(q.job + 1)) continue;
      Req* r = q.r;
      q.r = nullptr;
      r->result.assign(res_arena + q.out_off, res_arena + q.out_off + ((int64_t)1 << q.k));
      finish(r, QS_OK);   // r may be freed by its waiter from here on
      any = true;
    }
    while (!in_queue.empty() && !in_queue.front().r) in_queue.pop_front();
    op_tail = in_queue.empty() ? op_head : in_queue.front().op_start;
    res_tail = in_queue.empty() ? res_head : in_queue.front().res_start;
    return any;
  }

  qs_status launch_persistent() {
    QS_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), pk_stream));
    const int P = cfg.persistent_ctas;
    pk_reserved = std::min(P, sms / 2);
    g_reserved_sms.fetch_add(pk_reserved);
    const uint64_t idle_ns = (uint64_t)cfg.idle_ms * 1000000ull;
    if (cfg.prec == QS_C64)
      packed_persistent_kernel<float><<<P, 256, pk_smem, pk_stream>>>(
          ctl, jobs, reinterpret_cast<const PlainOp<float>*>(op_arena), res_arena, done_words, d_head,
          d_status, cfg.small_max_qubits, idle_ns, kLifeNs);
    else
      packed_persistent_kernel<double><<<P, 256, pk_smem, pk_stream>>>(
          ctl, jobs, reinterpret_cast<const PlainOp<double>*>(op_arena), res_arena, done_words, d_head,
          d_status, cfg.small_max_qubits, idle_ns, kLifeNs);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(pk_ev, pk_stream);
    if (e != cudaSuccess) {
      g_reserved_sms.fetch_sub(pk_reserved);
      pk_reserved = 0;
      return cuda_status(e, "persistent packed kernel launch");
    }
    pk_running = true;
    ++packed_launches;
    return QS_OK;
  }

  cudaError_t query(cudaEvent_t ev) {
    const int inj = injected_error.exchange(0);
    if (inj != 0) return (cudaError_t)inj;
    return cudaEventQuery(ev);
  }

  // fail every published job that is not finished and start the queue over
  void fail_queue(qs_status st, const std::string& msg) {
    for (QJob& q : in_queue)
      if (q.r) {
        Req* r = q.r;
        q.r = nullptr;
        set_error("%s", msg.c_str());
        finish(r, st);
      }
    in_queue.clear();
    op_tail = op_head;
    res_tail = res_head;
    cudaMemsetAsync(d_head, 0, sizeof(unsigned long long), pk_stream);
    cudaStreamSynchronize(pk_stream);
    published = 0;
    reinterpret_cast<std::atomic<uint64_t>*>(&ctl->tail)->store(0, std::memory_order_release);
  }

  // the persistent kernel has ended: by the idle limit (status QS_ETIMEOUT), its
  // lifetime, or an error; on an error its unfinished jobs fail with that error
  bool poll_persistent() {
    if (!pk_running) return false;
    const cudaError_t e = query(pk_ev);
    if (e == cudaErrorNotReady) return false;
    if (e != cudaSuccess) {
      cudaGetLastError();
      const qs_status st = cuda_status(e, "completion of the persistent packed kernel");
      const std::string msg = qs_last_error();
      cudaStreamSynchronize(pk_stream);   // nothing of it may still run when the queue starts over
      cudaGetLastError();
      pk_running = false;
      g_reserved_sms.fetch_sub(pk_reserved);
      pk_reserved = 0;
      fail_queue(st, msg);
      return true;
    }
    pk_running = false;
    g_reserved_sms.fetch_sub(pk_reserved);
    pk_reserved = 0;
    int status = 0;
    if (cudaMemcpy(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess &&
        status == (int)QS_ETIMEOUT) {
      std::lock_guard<std::mutex> g(mu);
      ++idle_timeouts;
    }
    return true;
  }

  // ---------------------------------------------------------------- large circuits
  void worker_loop() {
    cudaSetDevice(device);
    cudaStream_t stream = nullptr;
    cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    double* hbuf = nullptr;
    cudaMallocHost((void**)&hbuf, sizeof(double) << kMaxMargBits);
    const int method = cfg.large_tiled ? QS_METHOD_TILED : QS_METHOD_AUTO;
    for (;;) {
      Req* r = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_large.wait(lk, [&] { return stop_workers || !large_queue.empty(); });
        if (large_queue.empty()) break;
        r = large_queue.front();
        large_queue.pop_front();
        ++large_running;
      }
      qs_allocator a{async_alloc, async_free, nullptr};
      qs_state_t st = nullptr;
      qs_status s = (stream && hbuf) ? sv_create(r->n, cfg.prec, &a, stream, &st) : QS_ENOMEM;
      if (s == QS_OK)   // a host exception (planner allocation) fails this circuit, not the server
        s = abi_guard("large circuit", [&]() -> qs_status {
          qs_status s2 = apply_gates(st, r->gates.data(), r->gates.size(), method, nullptr);
          if (s2 != QS_OK) return s2;
          unsigned char* sc = (unsigned char*)st->scratch;
          double* marg = (double*)(sc + kScratchMarg);
          const bool all = r->k == r->n;   // a mask of all n bits is the plain distribution
          s2 = launch_probs(st, all ? marg : nullptr, 1, all ? 0 : r->mask, (double*)(sc + kScratchPartials),
                            (uint8_t*)(sc + kScratchBits), marg);
          if (s2 == QS_OK) {
            cudaError_t e = cudaMemcpyAsync(hbuf, marg, sizeof(double) << r->k, cudaMemcpyDeviceToHost, stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
            if (e != cudaSuccess) s2 = cuda_status(e, "large circuit readout");
          }
          if (s2 == QS_OK) r->result.assign(hbuf, hbuf + ((size_t)1 << r->k));
          return s2;
        });
      if (st) sv_destroy(st);
      {
        std::lock_guard<std::mutex> g(mu);
        bytes_in_use -= r->bytes;
        --large_running;
        ++large_circuits;
      }
      finish(r, s);
      cv_work.notify_one();
    }
    if (hbuf) cudaFreeHost(hbuf);
    if (stream) cudaStreamDestroy(stream);
  }

  // ---------------------------------------------------------------- scheduler
  void run() {
    cudaSetDevice(device);
    std::deque<Req*> small_wait;   // small circuits waiting for queue or arena space
    for (;;) {
      bool progress = retire_small();
      if (poll_persistent()) progress = true;
      std::vector<Req*> too_big;
      {
        std::lock_guard<std::mutex> g(mu);
        const bool idle = pending.empty() && small_wait.empty() && in_queue.empty() && !pk_running &&
                          large_queue.empty() && large_running == 0;
        if (stop && idle) return;
        for (auto it = pending.begin(); it != pending.end();) {
          Req* r = *it;
          if (r->n <= cfg.small_max_qubits) {
            small_wait.push_back(r);
            it = pending.erase(it);
            continue;
          }
          const size_t need = ((size_t)(cfg.prec == QS_C64 ? 8 : 16) << r->n) + kScratchBytes + (4u << 20);
          if (need > cfg.mem_budget) {   // can never be admitted
            too_big.push_back(r);
            it = pending.erase(it);
            continue;
          }
          if (bytes_in_use + need <= cfg.mem_budget &&
              (int)large_queue.size() + large_running < cfg.max_inflight) {
            r->bytes = need;
            bytes_in_use += need;
            peak_bytes = std::max(peak_bytes, bytes_in_use);
            large_queue.push_back(r);
            it = pending.erase(it);
            cv_large.notify_one();
            continue;
          }
          ++it;
        }
      }
      for (Req* r : too_big) {
        set_error("circuit of %d qubits needs more device memory than the server budget", r->n);
        finish(r, QS_ENOMEM);
        progress = true;
      }
      while (!small_wait.empty() && publish(small_wait.front())) {
        small_wait.pop_front();
        progress = true;
      }
      bool unfinished = false;
      for (const QJob& q : in_queue) unfinished = unfinished || q.r != nullptr;
      if (!pk_running && unfinished) {   // published jobs and no kernel to take them
        const qs_status s = launch_persistent();
        if (s != QS_OK) fail_queue(s, qs_last_error());
        progress = true;
      }
      if (!progress) {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait_for(lk, std::chrono::microseconds(10));
      }
    }
  }
};

}  // namespace qs

using namespace qs;

struct qs_server_s : public qs::Server {};

extern "C" {

qs_status qs_server_create(const qs_server_config* cfg, qs_server_t* out) {
  return abi_guard(__func__, [&]() -> qs_status {
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
        cfg->persistent_ctas < 0 || cfg->idle_ms < 0) {
      set_error("bad server configuration");
      return QS_EINVAL;
    }
    qs_server_s* s = new (std::nothrow) qs_server_s();
    if (!s) return QS_ENOMEM;
    s->cfg = *cfg;
    if (s->cfg.small_max_qubits == 0) s->cfg.small_max_qubits = small_cap;
    if (s->cfg.max_inflight == 0) s->cfg.max_inflight = 4;
    if (s->cfg.persistent_ctas == 0) s->cfg.persistent_ctas = 16;
    if (s->cfg.idle_ms == 0) s->cfg.idle_ms = 5;
    cudaGetDevice(&s->device);
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    if (s->cfg.persistent_ctas > s->sms) s->cfg.persistent_ctas = s->sms;
    if (s->cfg.mem_budget == 0) {
      size_t fr = 0, tot = 0;
      cudaMemGetInfo(&fr, &tot);
      s->cfg.mem_budget = (uint64_t)(0.8 * (double)fr);
    }
    // the persistent kernel's shared memory: the largest small state, the marginal
    // histogram and the op chunk
    const size_t amp = s->cfg.prec == QS_C64 ? sizeof(C2<float>) : sizeof(C2<double>);
    s->op_size = s->cfg.prec == QS_C64 ? sizeof(PlainOp<float>) : sizeof(PlainOp<double>);
    s->pk_smem = (amp << s->cfg.small_max_qubits) + (sizeof(double) << kMaxMargBits) + kOpChunk * s->op_size;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) {
      if (e == cudaSuccess) e = x;
    };
    chk(cudaStreamCreateWithFlags(&s->pk_stream, cudaStreamNonBlocking));
    chk(cudaEventCreateWithFlags(&s->pk_ev, cudaEventDisableTiming));
    const unsigned hflags = cudaHostAllocMapped | cudaHostAllocPortable;
    chk(cudaHostAlloc((void**)&s->ctl, sizeof(PCtl), hflags));
    chk(cudaHostAlloc((void**)&s->jobs, sizeof(PJob) * kRing, hflags));
    chk(cudaHostAlloc((void**)&s->done_words, sizeof(uint32_t) * kRing, hflags));
    chk(cudaHostAlloc((void**)&s->op_arena, s->op_size * (size_t)kOpArena, hflags));
    chk(cudaHostAlloc((void**)&s->res_arena, sizeof(double) * (size_t)kResArena, hflags));
    chk(cudaMalloc(&s->d_head, sizeof(unsigned long long)));
    chk(cudaMalloc(&s->d_status, sizeof(int)));
    if (e == cudaSuccess) {
      std::memset(s->ctl, 0, sizeof(PCtl));
      std::memset(s->done_words, 0, sizeof(uint32_t) * kRing);
      chk(cudaMemset(s->d_head, 0, sizeof(unsigned long long)));
      chk(cudaMemset(s->d_status, 0, sizeof(int)));
      if (s->cfg.prec == QS_C64)
        chk(cudaFuncSetAttribute(packed_persistent_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)s->pk_smem));
      else
        chk(cudaFuncSetAttribute(packed_persistent_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)s->pk_smem));
    }
    if (e != cudaSuccess) {
      qs_status st = cuda_status(e, "server setup");
      qs_server_destroy(s);
      return st;
    }
    s->scheduler = std::thread([s]() { s->run(); });
    for (int i = 0; i < s->cfg.max_inflight; ++i) s->workers.emplace_back([s]() { s->worker_loop(); });
    *out = s;
    return QS_OK;
  });
}

qs_status qs_server_submit(qs_server_t s, int n, const qs_gate* gates, size_t ngates,
                           uint64_t marg_mask, int64_t* ticket) {
  return abi_guard(__func__, [&]() -> qs_status {
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
  });
}

qs_status qs_server_wait(qs_server_t s, int64_t ticket, double* result, double* latency_ms) {
  return abi_guard(__func__, [&]() -> qs_status {
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
  });
}

qs_status qs_server_stats_get(qs_server_t s, qs_server_stats* out) {
  return abi_guard(__func__, [&]() -> qs_status {
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
    out->idle_timeouts = s->idle_timeouts;
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
  });
}

qs_status qs_server_inject_query_error(qs_server_t s, int cuda_error) {
  return abi_guard(__func__, [&]() -> qs_status {
    if (!s || cuda_error <= 0 || cuda_error == (int)cudaErrorNotReady) {
      set_error("server and a CUDA error code other than cudaErrorNotReady are required");
      return QS_EINVAL;
    }
    s->injected_error.store(cuda_error);
    return QS_OK;
  });
}

qs_status qs_server_destroy(qs_server_t s) {
  return abi_guard(__func__, [&]() -> qs_status {
    if (!s) return QS_OK;
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->scheduler.joinable()) s->scheduler.join();
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->stop_workers = true;
    }
    s->cv_large.notify_all();
    for (auto& w : s->workers)
      if (w.joinable()) w.join();
    if (s->ctl) reinterpret_cast<std::atomic<uint32_t>*>(&s->ctl->stop)->store(1u, std::memory_order_release);
    if (s->pk_stream) cudaStreamSynchronize(s->pk_stream);   // the kernel ends at its next wait
    if (s->pk_reserved) g_reserved_sms.fetch_sub(s->pk_reserved);
    for (auto& kv : s->reqs) delete kv.second;
    if (s->pk_stream) cudaStreamDestroy(s->pk_stream);
    if (s->pk_ev) cudaEventDestroy(s->pk_ev);
    if (s->ctl) cudaFreeHost(s->ctl);
    if (s->jobs) cudaFreeHost(s->jobs);
    if (s->done_words) cudaFreeHost(s->done_words);
    if (s->op_arena) cudaFreeHost(s->op_arena);
    if (s->res_arena) cudaFreeHost(s->res_arena);
    if (s->d_head) cudaFree(s->d_head);
    if (s->d_status) cudaFree(s->d_status);
    delete s;
    return QS_OK;
  });
}

}  // extern "C"
