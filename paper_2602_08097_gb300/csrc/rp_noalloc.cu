// rp_search_noalloc: GreedySearch for callers that must not allocate device
// memory.  Everything the kernel needs beyond the caller's inputs and outputs
// lives in one fixed array of this file, so the call makes no cudaMalloc,
// cudaMallocAsync or cudaFree and creates no context object.
//
// Who needs this: a serving process that reserves all of its device memory
// up front (an inference engine's memory pool, or an arena shared with other
// models) has nothing left for a library to allocate, and a caller that
// brackets its work in stream capture must not see allocations appear in its
// graph.  Both still own the vectors, the graph and the result buffers; they
// only cannot hand the library new memory per call.
#include <cstddef>
#include <mutex>

#include "internal.h"
#include "rp.h"

namespace {

// The whole scratch: the status word (offset 0) and the query counter
// (offset 128).  Every GPU that loads this library holds these
// RP_NOALLOC_SCRATCH_BYTES until exit.
constexpr size_t kHeader = 256;
static_assert(kHeader <= RP_NOALLOC_SCRATCH_BYTES, "scratch too small for its header");
static __device__ __align__(256) unsigned char g_noalloc_scratch[RP_NOALLOC_SCRATCH_BYTES];

// Device addresses of the array per device ordinal (in host code the symbol is
// only a host-side stand-in and must not be passed to a kernel).  The address
// is looked up again on every call made outside a stream capture, so a device
// reset between calls leaves no stale address behind; a call made while its
// stream captures uses the address the last uncaptured call on that device
// found.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

size_t elem_size(int dtype) { return dtype == RP_U8 ? 1 : 4; }

// The scratch array's device address on the current device (its ordinal in
// *dev_out), or nullptr if it cannot be had.
void* scratch_address(cudaStream_t stream, int* dev_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  *dev_out = dev;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return nullptr;
    g_scratch_addr[dev] = p;
  }
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" rp_status rp_search_noalloc(const void* vectors, int32_t dtype, int64_t n, int32_t d,
                                       const int64_t* row_ptr, const int32_t* col, int64_t start,
                                       const void* queries, int64_t nq, int32_t L, int32_t k, int32_t* ids,
                                       float* dists, void* cuda_stream) {
  if (dtype != RP_U8 && dtype != RP_F32) return RP_EINVAL;
  if (!vectors || !row_ptr || !col || !ids || (nq > 0 && !queries)) return RP_EINVAL;
  if (n < 1 || n > INT32_MAX || d < 1 || nq < 0 || k < 1 || L < k || L > RP_MAX_L) return RP_EINVAL;
  if (start < 0 || start >= n) return RP_EINVAL;
  const int64_t row_bytes = int64_t(d) * int64_t(elem_size(dtype));
  // the kernel reads rows with 16-byte loads
  if (row_bytes % 16 != 0 || reinterpret_cast<uintptr_t>(vectors) % 16 != 0 ||
      reinterpret_cast<uintptr_t>(queries) % 16 != 0)
    return RP_EINVAL;
  if (nq == 0) return RP_OK;

  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  void* base = scratch_address(stream, &dev);
  if (!base) return RP_ECUDA;
  int num_sms = 0;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RP_ECUDA;

  unsigned char* s = static_cast<unsigned char*>(base);
  rpk::DevStatus* status = reinterpret_cast<rpk::DevStatus*>(s);
  unsigned int* work = reinterpret_cast<unsigned int*>(s + 128);

  // The array keeps the last call's contents: the header must start at zero.
  if (cudaMemsetAsync(s, 0, kHeader, stream) != cudaSuccess) return RP_ECUDA;

  rpk::SearchLaunch S;
  S.data.X = static_cast<const uint8_t*>(vectors);
  S.data.row_bytes = row_bytes;
  S.data.n = n;
  S.data.d = d;
  S.data.dtype = dtype;
  S.row_ptr = row_ptr;
  S.col = col;
  S.start = start;
  S.Q = static_cast<const uint8_t*>(queries);
  S.nq = nq;
  S.L = L;
  S.k = k;
  S.out_ids = ids;
  S.out_dists = dists;
  S.num_sms = num_sms;
  S.work = work;
  S.status = status;
  return rpk::launch_search(S, stream) == cudaSuccess ? RP_OK : RP_ECUDA;
}

extern "C" rp_status rp_search_noalloc_status(void* cuda_stream, int64_t* info) {
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return RP_ECUDA;
  if (cap != cudaStreamCaptureStatusNone) return RP_EINVAL;  // it waits for the stream
  int dev = 0;
  void* base = scratch_address(stream, &dev);
  if (!base) return RP_ECUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return RP_ECUDA;
  rpk::DevStatus st;
  // the status word and its detail, read into this stack frame: nothing is allocated
  if (cudaMemcpy(&st, base, offsetof(rpk::DevStatus, fp64_decisions), cudaMemcpyDeviceToHost) != cudaSuccess)
    return RP_ECUDA;
  if (info) *info = st.info;
  return st.code == rpk::kDevOk ? RP_OK : RP_EDEVICE;
}
