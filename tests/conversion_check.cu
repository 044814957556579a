// Device check of the integer-only conversions of df.cuh against the
// conversion instructions: f2d_exact over every float bit pattern; d2f_rn
// over every double exponent with mantissas at and around the rounding
// boundary of every shift (and their complements and top-bit variants), and
// over 2^32 pseudo-random bit patterns (splitmix64), half of them with
// exponents near the float range.  NaNs are compared as NaN-ness only.
// Prints one JSON line with the mismatch counts.
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

#include "df.cuh"

namespace {

__device__ uint64_t splitmix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ void check_narrow(uint64_t u, unsigned long long* bad) {
  const double x = __longlong_as_double((long long)u);
  const float a = zbus::d2f_rn(x), b = __double2float_rn(x);
  if (!((a != a && b != b) || __float_as_uint(a) == __float_as_uint(b))) atomicAdd(bad, 1ull);
}

__global__ void k_widen(unsigned long long* bad) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (1ull << 32);
       i += (uint64_t)gridDim.x * blockDim.x) {
    const float f = __uint_as_float((uint32_t)i);
    const double a = zbus::f2d_exact(f), b = (double)f;
    if (!((a != a && b != b) || __double_as_longlong(a) == __double_as_longlong(b)))
      atomicAdd(bad, 1ull);
  }
}

// grid (2048 exponents, 2 signs), 64 threads: mantissas base + (t - 32) for
// base = 0 and 2^(s-1), s = 1..52
__global__ void k_narrow_edges(unsigned long long* bad) {
  const uint64_t ed = blockIdx.x, sg = (uint64_t)blockIdx.y << 63;
  const int t = threadIdx.x;
  for (int s = 0; s < 53; ++s) {
    const uint64_t base = s == 0 ? 0 : (1ull << (s - 1));
    const uint64_t m = (base + (uint64_t)(int64_t)(t - 32)) & 0xFFFFFFFFFFFFFull;
    check_narrow(sg | (ed << 52) | m, bad);
    check_narrow(sg | (ed << 52) | (m | 0x8000000000000ull), bad);
    check_narrow(sg | (ed << 52) | ((~m) & 0xFFFFFFFFFFFFFull), bad);
  }
}

__global__ void k_narrow_random(unsigned long long* bad, uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t u = splitmix(i);
    check_narrow(u, bad);
    const uint64_t ed = 1023 - 160 + (splitmix(u) % 300);
    check_narrow((u & 0x800FFFFFFFFFFFFFull) | (ed << 52), bad);
  }
}

}  // namespace

int main() {
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(unsigned long long)) != cudaSuccess) return 1;
  cudaMemset(d, 0, 2 * sizeof(unsigned long long));
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  k_widen<<<sms * 8, 256>>>(d);
  k_narrow_edges<<<dim3(2048, 2), 64>>>(d + 1);
  k_narrow_random<<<sms * 8, 256>>>(d + 1, 1ull << 31);
  const cudaError_t e = cudaDeviceSynchronize();
  unsigned long long h[2] = {~0ull, ~0ull};
  cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  std::printf("{\"status\": \"%s\", \"widen_mismatches\": %llu, \"narrow_mismatches\": %llu}\n",
              cudaGetErrorString(e), h[0], h[1]);
  return e == cudaSuccess ? 0 : 1;
}
