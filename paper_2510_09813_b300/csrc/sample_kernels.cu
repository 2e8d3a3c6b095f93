// Bitstring sampling from |psi_b|^2 (the measurement results an emulator returns,
// arXiv 2510.09813 Sec. III): b = min{ b : cdf(b) > u * cdf(D-1) }, with
// uniforms u from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), one
// counter per shot.
//
// The state is cut into chunks of kSampleChunk amplitudes. One warp sums each
// chunk; the exclusive prefix of the chunk sums is formed on the host in FP64.
// Each shot binary-searches that prefix, then runs through its chunk in index
// order. |psi_b|^2 and the running sums are FP64-class: for complex64 they are
// double words (exact squares by Dekker's FMA product, sums by Knuth's TwoSum)
// on the FP32 pipe, because FP64 instructions cost about 70 cycles of an SM
// sub-partition each on this part; complex128 uses FP64. Comparisons of the
// non-negative FP64 prefix against the target are made on the bit patterns as
// integers (the IEEE order of non-negative doubles).
#include <type_traits>

#include "dword.cuh"
#include "kernels.h"
#include "rsv_common.cuh"

namespace rsv {

// |psi_b|^2 as a double word (complex64) or a double (complex128).
__device__ __forceinline__ DW prob_dw(float re, float im) {
  const float a = __fmul_rn(re, re), b = __fmul_rn(im, im);
  const float ea = __fmaf_rn(re, re, -a), eb = __fmaf_rn(im, im, -b);
  float e;
  const float s = two_sum(a, b, e);
  return dw_renorm(s, __fadd_rn(e, __fadd_rn(ea, eb)));
}
__device__ __forceinline__ DW dw_add(DW x, DW y) {
  float e;
  const float s = two_sum(x.hi, y.hi, e);
  return dw_renorm(s, __fadd_rn(e, __fadd_rn(x.lo, y.lo)));
}

template <typename Real>
__device__ __forceinline__ double prob_at(const void* psi, int64_t b) {
  using C = typename CplxT<Real>::type;
  const C v = reinterpret_cast<const C*>(psi)[b];
  const double re = (double)v.x, im = (double)v.y;
  return re * re + im * im;
}

// One warp per chunk: lane l takes amplitudes l, l + 32, ... of the chunk
// (coalesced); the warp's sums are combined in a fixed tree.
template <typename Real>
__global__ void chunk_sum_kernel(const void* psi, int64_t dim, int64_t chunk, double* sums) {
  const int64_t nchunks = (dim + chunk - 1) / chunk;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= nchunks) return;
  const int64_t lo = c * chunk, hi = lo + chunk < dim ? lo + chunk : dim;
  if constexpr (std::is_same<Real, float>::value) {
    const float2* p = reinterpret_cast<const float2*>(psi);
    DW acc{0.f, 0.f};
    for (int64_t b = lo + lane; b < hi; b += 32) {
      const float2 v = p[b];
      acc = dw_add(acc, prob_dw(v.x, v.y));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
      acc = dw_add(acc, DW{__shfl_xor_sync(0xffffffffu, acc.hi, off), __shfl_xor_sync(0xffffffffu, acc.lo, off)});
    if (lane == 0) sums[c] = dw_value(acc);
  } else {
    double acc = 0.0;
    for (int64_t b = lo + lane; b < hi; b += 32) acc += prob_at<Real>(psi, b);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) sums[c] = acc;
  }
}

__device__ __forceinline__ void philox_round(uint32_t (&x)[4], uint32_t k0, uint32_t k1) {
  const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
  const uint32_t hi0 = __umulhi(m0, x[0]), lo0 = m0 * x[0];
  const uint32_t hi1 = __umulhi(m1, x[2]), lo1 = m1 * x[2];
  const uint32_t y0 = hi1 ^ x[1] ^ k0, y1 = lo1, y2 = hi0 ^ x[3] ^ k1, y3 = lo0;
  x[0] = y0;
  x[1] = y1;
  x[2] = y2;
  x[3] = y3;
}

__device__ __forceinline__ double shot_uniform(uint64_t seed, uint64_t shot) {
  uint32_t x[4] = {(uint32_t)shot, (uint32_t)(shot >> 32), 0u, 0u};
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    philox_round(x, k0, k1);
  }
  const uint64_t u53 = ((uint64_t)x[0] << 21) | (uint64_t)(x[1] >> 11);
  return (double)u53 * 0x1.0p-53;
}

// a <= b for non-negative doubles, on their bit patterns
__device__ __forceinline__ bool le_nonneg(double a, double b) {
  return __double_as_longlong(a) <= __double_as_longlong(b);
}

template <typename Real>
__global__ void sample_kernel(const void* psi, int64_t dim, int64_t chunk, const double* chunk_cdf, int64_t nchunks,
                              double total, int64_t shots, uint64_t seed, uint64_t* out) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= shots) return;
  const double target = shot_uniform(seed, (uint64_t)s) * total;
  // last chunk whose exclusive prefix is <= target
  int64_t lo = 0, hi = nchunks - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (le_nonneg(chunk_cdf[mid], target)) lo = mid;
    else hi = mid - 1;
  }
  const int64_t b0 = lo * chunk, b1 = b0 + chunk < dim ? b0 + chunk : dim;
  int64_t pick = -1, last_nonzero = -1;
  if constexpr (std::is_same<Real, float>::value) {
    // run > target  <=>  (run - prefix) > (target - prefix), in double words
    const DW need = dw_from(target - chunk_cdf[lo]);
    const float2* p = reinterpret_cast<const float2*>(psi);
    DW run{0.f, 0.f};
    for (int64_t b = b0; b < b1; ++b) {
      const float2 v = p[b];
      if (v.x != 0.f || v.y != 0.f) last_nonzero = b;
      run = dw_add(run, prob_dw(v.x, v.y));
      if (run.hi > need.hi || (run.hi == need.hi && run.lo > need.lo)) {
        pick = b;
        break;
      }
    }
  } else {
    double run = chunk_cdf[lo];
    for (int64_t b = b0; b < b1; ++b) {
      const double pb = prob_at<Real>(psi, b);
      run += pb;
      if (pb > 0.0) last_nonzero = b;
      if (run > target) {
        pick = b;
        break;
      }
    }
  }
  if (pick < 0) pick = last_nonzero >= 0 ? last_nonzero : (b1 - 1);
  out[s] = (uint64_t)pick;
}

cudaError_t launch_block_sums(const void* psi, int64_t dim, bool c64, int64_t chunk, double* sums, cudaStream_t stream) {
  const int64_t nchunks = (dim + chunk - 1) / chunk;
  const int threads = 256;  // 8 chunks per block, one warp each
  const int64_t blocks = (nchunks + threads / 32 - 1) / (threads / 32);
  if (c64)
    chunk_sum_kernel<float><<<(unsigned)blocks, threads, 0, stream>>>(psi, dim, chunk, sums);
  else
    chunk_sum_kernel<double><<<(unsigned)blocks, threads, 0, stream>>>(psi, dim, chunk, sums);
  return cudaGetLastError();
}

cudaError_t launch_sample(const void* psi, int64_t dim, bool c64, int64_t chunk, const double* chunk_cdf, int64_t nchunks,
                          double total, int64_t shots, uint64_t seed, uint64_t* out, cudaStream_t stream) {
  const int threads = 128;
  const int64_t blocks = (shots + threads - 1) / threads;
  if (blocks == 0) return cudaSuccess;
  if (c64)
    sample_kernel<float><<<(unsigned)blocks, threads, 0, stream>>>(psi, dim, chunk, chunk_cdf, nchunks, total, shots,
                                                                    seed, out);
  else
    sample_kernel<double><<<(unsigned)blocks, threads, 0, stream>>>(psi, dim, chunk, chunk_cdf, nchunks, total, shots,
                                                                     seed, out);
  return cudaGetLastError();
}

}  // namespace rsv
