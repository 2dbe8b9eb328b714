// alpha-reachability of a graph (Definition 2.1), per node.
//
// For a node p the term is
//   min over q != p with (p, q) not an edge of  max over p' in N_out(p) of D(p, q) / D(p', q),
// with D(p', q) = 0 giving +inf (q is reachable at every alpha), a node without
// out-neighbours giving 0, and no such q giving +inf; alpha*(G) is the minimum
// of the terms over all nodes.  A graph is alpha-reachable exactly when alpha
// is at most alpha*(G).
//
// Arithmetic: uint8 squared distances are exact integers; float32 ones are the
// canonical binary64 difference form (index order, no fused multiply-add);
// D = sqrt(d2) and the ratio are IEEE binary64, so every term is bit-exact.
//
// One CTA per node asked for; its threads stride over every q.  A q whose
// running maximum already reaches the CTA's running minimum cannot lower it,
// so its scan over N_out(p) stops there (the minimum, and with it the term, is
// unchanged); the CTA's minimum is shared through its bit pattern, which
// orders non-negative doubles as unsigned integers.
#include <cmath>

#include "internal.h"

namespace rpk {

namespace {

template <int DT>
__device__ __forceinline__ double exact_d2(const uint8_t* __restrict__ a, const uint8_t* __restrict__ b,
                                           int64_t row_bytes, int d) {
  if constexpr (DT == kU8) {
    const uint4* pa = reinterpret_cast<const uint4*>(a);
    const uint4* pb = reinterpret_cast<const uint4*>(b);
    unsigned acc = 0;  // below 2^32 for d <= 65536
    for (int64_t c = 0; c < row_bytes / 16; ++c) {
      const uint4 x = __ldg(pa + c), y = __ldg(pb + c);
      acc = sqdiff4_u8(x.x, y.x, acc);
      acc = sqdiff4_u8(x.y, y.y, acc);
      acc = sqdiff4_u8(x.z, y.z, acc);
      acc = sqdiff4_u8(x.w, y.w, acc);
    }
    return double(acc);
  } else {
    return canon_d2_f32(reinterpret_cast<const float*>(a), reinterpret_cast<const float*>(b), d);
  }
}

template <int DT>
__global__ void __launch_bounds__(256) reach_kernel(DevData D, const int64_t* __restrict__ row_ptr,
                                                    const int32_t* __restrict__ col,
                                                    const int64_t* __restrict__ nodes, int64_t n_nodes,
                                                    double* __restrict__ out) {
  __shared__ unsigned long long s_min;  // bit pattern of the CTA's running minimum
  for (int64_t i = blockIdx.x; i < n_nodes; i += gridDim.x) {
    const int64_t p = nodes ? nodes[i] : i;
    if (threadIdx.x == 0) s_min = __double_as_longlong(INFINITY);
    __syncthreads();
    const int64_t e0 = row_ptr[p], e1 = row_ptr[p + 1];
    const uint8_t* xp = D.X + p * D.row_bytes;
    for (int64_t q = threadIdx.x; q < D.n; q += blockDim.x) {
      if (q == p) continue;
      const double cur = __longlong_as_double(*reinterpret_cast<volatile unsigned long long*>(&s_min));
      const uint8_t* xq = D.X + q * D.row_bytes;
      const double dpq = __dsqrt_rn(exact_d2<DT>(xp, xq, D.row_bytes, D.d));
      double best = 0.0;
      bool skip = false;  // q is an out-neighbour, or cannot lower the minimum
      for (int64_t e = e0; e < e1; ++e) {
        const int32_t v = col[e];
        if (v == q) {
          skip = true;
          break;
        }
        const double dd = __dsqrt_rn(exact_d2<DT>(D.X + int64_t(v) * D.row_bytes, xq, D.row_bytes, D.d));
        const double r = dd == 0.0 ? INFINITY : __ddiv_rn(dpq, dd);
        if (r > best) best = r;
        if (best >= cur) {
          skip = true;
          break;
        }
      }
      if (!skip && best < cur) atomicMin(&s_min, static_cast<unsigned long long>(__double_as_longlong(best)));
    }
    __syncthreads();
    if (threadIdx.x == 0) out[i] = __longlong_as_double(s_min);
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_reach(const DevData& D, const int64_t* row_ptr, const int32_t* col, const int64_t* nodes,
                         int64_t n_nodes, double* out, cudaStream_t s) {
  if (n_nodes <= 0) return cudaSuccess;
  const unsigned grid = unsigned(n_nodes < (int64_t(1) << 16) ? n_nodes : (int64_t(1) << 16));
  if (D.dtype == kF32) reach_kernel<kF32><<<grid, 256, 0, s>>>(D, row_ptr, col, nodes, n_nodes, out);
  else reach_kernel<kU8><<<grid, 256, 0, s>>>(D, row_ptr, col, nodes, n_nodes, out);
  return cudaGetLastError();
}

}  // namespace rpk
