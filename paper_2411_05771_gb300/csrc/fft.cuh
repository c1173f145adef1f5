// Radix-2 Stockham FFT in shared memory, shared by the Ram-Lak filter's
// FFT form and the multi-coil MRI operators.
#pragma once
#include "common.cuh"

namespace skei {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// tw[t] = e^{-2 pi i t / N}, t < N/2, into shared memory (no barrier).
__device__ __forceinline__ void twiddles(float2 *tw, int N) {
  for (int t = threadIdx.x; t < N / 2; t += blockDim.x) {
    float s, c;
    sincospif(2.0f * (float)t / (float)N, &s, &c);
    tw[t] = make_float2(c, -s);
  }
}

// Radix-2 Stockham FFT of cnt independent length-N sequences in shared
// memory: element i of sequence s at a[s ld_s + i ld_i]; b is scratch of the
// same shape.  inv: e^{+2 pi i ...} (unnormalised).  Thread t takes sequence
// t % cnt (s_fast) or t / (N/2).  Ends with a barrier; returns the buffer
// holding the result (a or b).
__device__ __forceinline__ float2 *fft_smem(float2 *a, float2 *b, int N, int cnt, int ld_s,
                                            int ld_i, const float2 *tw, bool inv, bool s_fast) {
  const int half = N / 2;
  for (int Ns = 1; Ns < N; Ns *= 2) {
    const int tstep = N / (2 * Ns);
    for (int t = threadIdx.x; t < cnt * half; t += blockDim.x) {
      const int s = s_fast ? t % cnt : t / half;
      const int j = s_fast ? t / cnt : t % half;
      const int k = j & (Ns - 1);
      float2 w = tw[k * tstep];
      if (inv) w.y = -w.y;
      const float2 u = a[s * ld_s + j * ld_i];
      const float2 v = cmul(a[s * ld_s + (j + half) * ld_i], w);
      const int o = 2 * j - k;   // (j / Ns) 2 Ns + k
      b[s * ld_s + o * ld_i] = make_float2(u.x + v.x, u.y + v.y);
      b[s * ld_s + (o + Ns) * ld_i] = make_float2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
    float2 *t = a;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace skei
