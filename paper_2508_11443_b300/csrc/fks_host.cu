// fks_host.cu -- builds and lookups over host buffers: the end-to-end path of
// a caller whose keys, needles and results live in host memory.  Built on
// the device entry points of fks_api.cu through the public ABI only.
//
// A lookup streams the needles through the device in chunks: chunk i is
// uploaded on one stream while chunk i - 1 is looked up on the caller's
// stream and the results of chunk i - 2 go back on a third, so the two
// directions of the host link and the lookup kernel overlap.  With pinned
// host buffers the copies are asynchronous DMA; pageable buffers work too,
// at the speed of the driver's staged copies.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "fks.h"

namespace {

constexpr uint64_t kChunk = 1ull << 23;  // needles per pipeline chunk
constexpr int kBuffers = 3;

struct HostPipe {
  cudaStream_t up = nullptr, down = nullptr;
  cudaEvent_t uploaded[kBuffers] = {}, looked[kBuffers] = {}, freed[kBuffers] = {};
  bool ok = false;
  HostPipe() {
    ok = cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; b < kBuffers && ok; ++b)
      ok = cudaEventCreateWithFlags(&uploaded[b], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&looked[b], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&freed[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) cudaGetLastError();
  }
  ~HostPipe() {
    for (int b = 0; b < kBuffers; ++b) {
      if (uploaded[b]) cudaEventDestroy(uploaded[b]);
      if (looked[b]) cudaEventDestroy(looked[b]);
      if (freed[b]) cudaEventDestroy(freed[b]);
    }
    if (up) cudaStreamDestroy(up);
    if (down) cudaStreamDestroy(down);
  }
};
thread_local HostPipe* g_pipe = nullptr;  // per host thread, created on first use

fks_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return FKS_OK;
  cudaGetLastError();
  return FKS_ERR_CUDA;
}

}  // namespace

extern "C" {

fks_status fks_build_u64_host(const uint64_t* h_keys, const void* h_vals, fks_val_type val_type, uint64_t n,
                              uint64_t seed, const fks_build_opts* opts, const fks_allocator* alloc,
                              fks_stream_t stream, fks_map_t* out) {
  if (!out) return FKS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!h_keys || !h_vals || n == 0 || n >= (1ull << 30) || (val_type != FKS_VAL_I32 && val_type != FKS_VAL_I64))
    return FKS_ERR_INVALID_ARG;
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t vb = val_type == FKS_VAL_I64 ? 8 : 4;
  uint8_t* d = nullptr;
  const size_t kb = (8 * n + 255) & ~size_t(255);
  if (cudaMallocAsync(reinterpret_cast<void**>(&d), kb + vb * n, st) != cudaSuccess) {
    cudaGetLastError();
    return FKS_ERR_OUT_OF_MEMORY;
  }
  fks_status s = cuda_status(cudaMemcpyAsync(d, h_keys, 8 * n, cudaMemcpyHostToDevice, st));
  if (s == FKS_OK) s = cuda_status(cudaMemcpyAsync(d + kb, h_vals, vb * n, cudaMemcpyHostToDevice, st));
  if (s == FKS_OK)  // the map keeps its own tables: the uploaded inputs are freed afterwards
    s = fks_build_u64(reinterpret_cast<const uint64_t*>(d), d + kb, val_type, n, seed, opts, alloc, stream, out);
  cudaFreeAsync(d, st);
  return s;
}

fks_status fks_lookup_u64_host(fks_map_t map, const uint64_t* h_q, uint64_t nq, void* h_out, uint8_t* h_found,
                               int64_t absent, fks_stream_t stream) {
  if (!map) return FKS_ERR_INVALID_ARG;
  if (nq == 0) return FKS_OK;
  if (!h_q) return FKS_ERR_INVALID_ARG;
  fks_map_info_t info;
  fks_status s = fks_map_info(map, &info);
  if (s != FKS_OK) return s;
  if (info.key_kind != FKS_KEY_U64) return FKS_ERR_INVALID_ARG;
  if (!g_pipe) g_pipe = new HostPipe();
  HostPipe& P = *g_pipe;
  if (!P.ok) return FKS_ERR_CUDA;
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t vb = info.val_type == FKS_VAL_I64 ? 8 : 4;
  const uint64_t C = nq < kChunk ? nq : kChunk;
  const size_t per = 8 * C + vb * C + C;  // needles, values, found flags of one buffer
  uint8_t* dev = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&dev), kBuffers * ((per + 255) & ~size_t(255)), st) != cudaSuccess) {
    cudaGetLastError();
    return FKS_ERR_OUT_OF_MEMORY;
  }
  // the buffers exist once the allocation on `st` is done
  cudaEvent_t ready = P.freed[0];
  s = cuda_status(cudaEventRecord(ready, st));
  if (s == FKS_OK) s = cuda_status(cudaStreamWaitEvent(P.up, ready, 0));
  for (int b = 1; b < kBuffers && s == FKS_OK; ++b) s = cuda_status(cudaEventRecord(P.freed[b], st));
  const uint64_t chunks = (nq + C - 1) / C;
  for (uint64_t i = 0; i < chunks && s == FKS_OK; ++i) {
    const int b = int(i % kBuffers);
    uint8_t* base = dev + size_t(b) * ((per + 255) & ~size_t(255));
    uint64_t* dq = reinterpret_cast<uint64_t*>(base);
    uint8_t* dv = base + 8 * C;
    uint8_t* df = dv + vb * C;
    const uint64_t q0 = i * C, cnt = nq - q0 < C ? nq - q0 : C;
    // upload, after the buffer's previous results went back
    s = cuda_status(cudaStreamWaitEvent(P.up, P.freed[b], 0));
    if (s == FKS_OK) s = cuda_status(cudaMemcpyAsync(dq, h_q + q0, 8 * cnt, cudaMemcpyHostToDevice, P.up));
    if (s == FKS_OK) s = cuda_status(cudaEventRecord(P.uploaded[b], P.up));
    // look up on the caller's stream
    if (s == FKS_OK) s = cuda_status(cudaStreamWaitEvent(st, P.uploaded[b], 0));
    if (s == FKS_OK) s = fks_lookup_u64(map, dq, cnt, h_out ? dv : nullptr, h_found ? df : nullptr, absent, stream);
    if (s == FKS_OK) s = cuda_status(cudaEventRecord(P.looked[b], st));
    // results back
    if (s == FKS_OK) s = cuda_status(cudaStreamWaitEvent(P.down, P.looked[b], 0));
    if (s == FKS_OK && h_out)
      s = cuda_status(cudaMemcpyAsync(static_cast<uint8_t*>(h_out) + vb * q0, dv, vb * cnt, cudaMemcpyDeviceToHost,
                                      P.down));
    if (s == FKS_OK && h_found)
      s = cuda_status(cudaMemcpyAsync(h_found + q0, df, cnt, cudaMemcpyDeviceToHost, P.down));
    if (s == FKS_OK) s = cuda_status(cudaEventRecord(P.freed[b], P.down));
  }
  // the caller's stream frees the buffers once the last results are back
  cudaStreamWaitEvent(st, P.freed[(chunks - 1) % kBuffers], 0);
  cudaFreeAsync(dev, st);
  const cudaError_t e = cudaStreamSynchronize(P.down);
  if (s == FKS_OK) s = cuda_status(e);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  if (s == FKS_OK) s = cuda_status(e2);
  return s;
}

}  // extern "C"
