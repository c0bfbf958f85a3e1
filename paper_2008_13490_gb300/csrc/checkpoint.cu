// Binary checkpoint of a state vector, for resuming an interrupted simulation
// (the thesis's solver saves its current state vector in binary form for
// exactly that).
//
// File: a 48-byte little-endian header
//   char     magic[8]   "QSIMSV1"
//   uint32   n          qubits
//   uint32   prec       QS_C64 / QS_C128
//   uint64   bytes      amplitude bytes (2^n x 8 or 16)
//   uint64   checksum   see below
//   uint64   reserved[2] (zero)
// followed by the 2^n interleaved (re, im) amplitudes in the state's precision.
//
// Checksum: over the amplitude bytes as 64-bit words w_i, the sum mod 2^64 of
// mix(w_i + (i + 1) * 0x9E3779B97F4A7C15) with mix the SplitMix64 finaliser
// (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
// 2014).  A sum is order-independent, so the GPU computes it with atomics and
// gets the same value every time.
//
// Both directions stream through two pinned host buffers: the device<->host copy
// of one chunk overlaps the file I/O of the other.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

#include "abi_guard.h"
#include "internal.h"

namespace qs {
namespace {

constexpr char kMagic[8] = {'Q', 'S', 'I', 'M', 'S', 'V', '1', '\0'};
constexpr size_t kChunk = size_t(64) << 20;   // bytes per pinned buffer

struct SvHeader {
  char magic[8];
  uint32_t n;
  uint32_t prec;
  uint64_t bytes;
  uint64_t checksum;
  uint64_t reserved[2];
};
static_assert(sizeof(SvHeader) == 48, "header layout");

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void __launch_bounds__(256)
    checksum_kernel(const uint64_t* __restrict__ w, uint64_t nwords, unsigned long long* __restrict__ out) {
  uint64_t acc = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nwords;
       i += (uint64_t)gridDim.x * blockDim.x)
    acc += mix64(__ldcs(w + i) + (i + 1) * 0x9E3779B97F4A7C15ull);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, (unsigned long long)acc);
}

qs_status device_checksum(State* st, uint64_t* sum) {
  unsigned long long* d = (unsigned long long*)((unsigned char*)st->scratch + kScratchResult);
  QS_CUDA(cudaMemsetAsync(d, 0, sizeof(*d), st->stream));
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t nwords = st->data_bytes / 8;
  uint64_t blocks = (nwords + 255) / 256;
  if (blocks > (uint64_t)sms * 8) blocks = (uint64_t)sms * 8;
  checksum_kernel<<<(unsigned)blocks, 256, 0, st->stream>>>((const uint64_t*)st->data, nwords, d);
  QS_CUDA(cudaGetLastError());
  QS_CUDA(cudaMemcpyAsync(sum, d, sizeof(*sum), cudaMemcpyDeviceToHost, st->stream));
  QS_CUDA(cudaStreamSynchronize(st->stream));
  return QS_OK;
}

struct Pinned {
  void* buf[2] = {nullptr, nullptr};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  ~Pinned() {
    for (int i = 0; i < 2; ++i) {
      if (ev[i]) {
        cudaEventSynchronize(ev[i]);
        cudaEventDestroy(ev[i]);
      }
      if (buf[i]) cudaFreeHost(buf[i]);
    }
  }
  qs_status init() {
    for (int i = 0; i < 2; ++i) {
      if (cudaHostAlloc(&buf[i], kChunk, cudaHostAllocDefault) != cudaSuccess) {
        buf[i] = nullptr;
        set_error("pinned staging allocation failed");
        return QS_ENOMEM;
      }
      QS_CUDA(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
    }
    return QS_OK;
  }
};

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" qs_status sv_save(qs_state_t h, const char* path) {
  return abi_guard(__func__, [&]() -> qs_status {
    State* st = h;
    if (!st || !path) {
      set_error("state and path are required");
      return QS_EINVAL;
    }
    SvHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, kMagic, 8);
    hd.n = (uint32_t)st->n;
    hd.prec = (uint32_t)st->prec;
    hd.bytes = st->data_bytes;
    qs_status s = device_checksum(st, &hd.checksum);
    if (s != QS_OK) return s;
    Pinned pin;
    s = pin.init();
    if (s != QS_OK) return s;
    File file;
    file.f = std::fopen(path, "wb");
    if (!file.f) {
      set_error("cannot open %s for writing", path);
      return QS_EINVAL;
    }
    if (std::fwrite(&hd, sizeof(hd), 1, file.f) != 1) {
      set_error("write to %s failed", path);
      return QS_EINVAL;
    }
    const unsigned char* src = (const unsigned char*)st->data;
    const size_t total = st->data_bytes, nchunks = (total + kChunk - 1) / kChunk;
    auto issue = [&](size_t c) -> qs_status {
      const size_t off = c * kChunk, len = total - off < kChunk ? total - off : kChunk;
      QS_CUDA(cudaMemcpyAsync(pin.buf[c & 1], src + off, len, cudaMemcpyDeviceToHost, st->stream));
      QS_CUDA(cudaEventRecord(pin.ev[c & 1], st->stream));
      return QS_OK;
    };
    if (nchunks) s = issue(0);
    for (size_t c = 0; c < nchunks && s == QS_OK; ++c) {
      if (c + 1 < nchunks) s = issue(c + 1);   // the next copy runs while this chunk is written
      if (s != QS_OK) break;
      QS_CUDA(cudaEventSynchronize(pin.ev[c & 1]));
      const size_t off = c * kChunk, len = total - off < kChunk ? total - off : kChunk;
      if (std::fwrite(pin.buf[c & 1], 1, len, file.f) != len) {
        set_error("write to %s failed", path);
        s = QS_EINVAL;
      }
    }
    if (s == QS_OK && std::fflush(file.f) != 0) {
      set_error("write to %s failed", path);
      s = QS_EINVAL;
    }
    // a late write error (full disk, network file system) shows up at close
    const int closed = std::fclose(file.f);
    file.f = nullptr;
    if (s == QS_OK && closed != 0) {
      set_error("closing %s failed: the checkpoint may be incomplete", path);
      s = QS_EINVAL;
    }
    return s;
  });
}

extern "C" qs_status sv_load(qs_state_t h, const char* path) {
  return abi_guard(__func__, [&]() -> qs_status {
    State* st = h;
    if (!st || !path) {
      set_error("state and path are required");
      return QS_EINVAL;
    }
    File file;
    file.f = std::fopen(path, "rb");
    if (!file.f) {
      set_error("cannot open %s", path);
      return QS_EINVAL;
    }
    SvHeader hd;
    if (std::fread(&hd, sizeof(hd), 1, file.f) != 1 || std::memcmp(hd.magic, kMagic, 8) != 0) {
      set_error("%s is not a state checkpoint", path);
      return QS_EINVAL;
    }
    if ((int)hd.n != st->n || (int)hd.prec != st->prec || hd.bytes != st->data_bytes) {
      set_error("checkpoint holds n = %u, prec = %u; the state has n = %d, prec = %d", hd.n, hd.prec,
                st->n, st->prec);
      return QS_EINVAL;
    }
    Pinned pin;
    qs_status s = pin.init();
    if (s != QS_OK) return s;
    unsigned char* dst = (unsigned char*)st->data;
    const size_t total = st->data_bytes, nchunks = (total + kChunk - 1) / kChunk;
    bool short_read = false;
    for (size_t c = 0; c < nchunks && s == QS_OK; ++c) {
      // the copy that last used this buffer (chunk c - 2) must have finished
      if (c >= 2) QS_CUDA(cudaEventSynchronize(pin.ev[c & 1]));
      const size_t off = c * kChunk, len = total - off < kChunk ? total - off : kChunk;
      if (std::fread(pin.buf[c & 1], 1, len, file.f) != len) {
        short_read = true;
        break;
      }
      QS_CUDA(cudaMemcpyAsync(dst + off, pin.buf[c & 1], len, cudaMemcpyHostToDevice, st->stream));
      QS_CUDA(cudaEventRecord(pin.ev[c & 1], st->stream));
    }
    QS_CUDA(cudaStreamSynchronize(st->stream));
    uint64_t sum = 0;
    if (s == QS_OK && !short_read) s = device_checksum(st, &sum);
    if (s == QS_OK && (short_read || sum != hd.checksum)) {
      // a partly loaded state must not pass for the checkpoint
      launch_set_basis(st, 0);
      cudaStreamSynchronize(st->stream);
      set_error(short_read ? "%s is truncated; the state was reset to |0...0>"
                           : "checksum mismatch in %s; the state was reset to |0...0>",
                path);
      return QS_EINVAL;
    }
    return s;
  });
}
