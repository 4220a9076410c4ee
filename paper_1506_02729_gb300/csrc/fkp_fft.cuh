// fkp_fft.cuh - batched shared-memory FFT building blocks for sm_103a.
//
// A batch of complex pencils of length n (n = 2^a 3^b 5^c <= 512) lives in
// shared memory, pencil p at base + p*stride.  Each radix stage reads one
// buffer and writes the other (self-sorting Stockham order, so the result is
// in natural order without a bit-reversal pass).  For a stage of radix R
// after stages whose radices multiply to ns, butterfly j (0 <= j < n/R)
// reads x[j + r n/R], multiplies by w^(r k n/(ns R)) with k = j mod ns,
// applies the length-R DFT and writes y[(j/ns) ns R + k + r ns].  Twiddles
// w^m = exp(-2 pi i m/n) come from a table computed in FP64 on the host and
// rounded to FP32.  DIR = -1 is the forward transform (sign e^{-ik.x}, the
// sign of eqs. deltaell and Qij), DIR = +1 the unnormalised inverse (the
// sign of eq. F_k).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fkp {

struct FftPlan {
  int n;
  int nst;
  int radix[8];
};

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by i*DIR  (i for DIR=+1, -i for DIR=-1)
template <int DIR>
__device__ __forceinline__ float2 mul_idir(float2 a) {
  return DIR > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Constants of the small DFTs (plain trigonometric values).
#define FKP_SQRT1_2 0.70710678118654752440f
#define FKP_SIN60 0.86602540378443864676f
#define FKP_C1_5 0.30901699437494742410f   // cos(2 pi/5)
#define FKP_C2_5 (-0.80901699437494742410f) // cos(4 pi/5)
#define FKP_S1_5 0.95105651629515357212f   // sin(2 pi/5)
#define FKP_S2_5 0.58778525229247312917f   // sin(4 pi/5)

template <int DIR>
__device__ __forceinline__ void dft2(float2* v) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <int DIR>
__device__ __forceinline__ void dft3(float2* v) {
  float2 t1 = cadd(v[1], v[2]);
  float2 t2 = make_float2(v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y);
  float2 t3 = mul_idir<DIR>(cscale(csub(v[1], v[2]), FKP_SIN60));
  v[0] = cadd(v[0], t1);
  v[1] = cadd(t2, t3);
  v[2] = csub(t2, t3);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2* v) {
  float2 s0 = cadd(v[0], v[2]), d0 = csub(v[0], v[2]);
  float2 s1 = cadd(v[1], v[3]), d1 = mul_idir<DIR>(csub(v[1], v[3]));
  v[0] = cadd(s0, s1);
  v[2] = csub(s0, s1);
  v[1] = cadd(d0, d1);
  v[3] = csub(d0, d1);
}

template <int DIR>
__device__ __forceinline__ void dft5(float2* v) {
  float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  float2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
  float2 a1 = make_float2(v[0].x + FKP_C1_5 * t1.x + FKP_C2_5 * t2.x, v[0].y + FKP_C1_5 * t1.y + FKP_C2_5 * t2.y);
  float2 a2 = make_float2(v[0].x + FKP_C2_5 * t1.x + FKP_C1_5 * t2.x, v[0].y + FKP_C2_5 * t1.y + FKP_C1_5 * t2.y);
  float2 b1 = mul_idir<DIR>(make_float2(FKP_S1_5 * t3.x + FKP_S2_5 * t4.x, FKP_S1_5 * t3.y + FKP_S2_5 * t4.y));
  float2 b2 = mul_idir<DIR>(make_float2(FKP_S2_5 * t3.x - FKP_S1_5 * t4.x, FKP_S2_5 * t3.y - FKP_S1_5 * t4.y));
  v[0] = cadd(v[0], cadd(t1, t2));
  v[1] = cadd(a1, b1);
  v[4] = csub(a1, b1);
  v[2] = cadd(a2, b2);
  v[3] = csub(a2, b2);
}

// Length-8 DFT as a radix-2 split: even outputs are the length-4 DFT of
// a_r + a_{r+4}; odd outputs the length-4 DFT of (a_r - a_{r+4}) w8^r.
template <int DIR>
__device__ __forceinline__ void dft8(float2* v) {
  float2 b[4], c[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    b[r] = cadd(v[r], v[r + 4]);
    c[r] = csub(v[r], v[r + 4]);
  }
  // c_r *= exp(DIR * 2 pi i r / 8)
  c[1] = make_float2(FKP_SQRT1_2 * (c[1].x - DIR * c[1].y), FKP_SQRT1_2 * (c[1].y + DIR * c[1].x));
  c[2] = mul_idir<DIR>(c[2]);
  c[3] = make_float2(FKP_SQRT1_2 * (-c[3].x - DIR * c[3].y), FKP_SQRT1_2 * (-c[3].y + DIR * c[3].x));
  dft4<DIR>(b);
  dft4<DIR>(c);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    v[2 * m] = b[m];
    v[2 * m + 1] = c[m];
  }
}

template <int R, int DIR>
__device__ __forceinline__ void dftR(float2* v) {
  if (R == 2) dft2<DIR>(v);
  else if (R == 3) dft3<DIR>(v);
  else if (R == 4) dft4<DIR>(v);
  else if (R == 5) dft5<DIR>(v);
  else dft8<DIR>(v);
}

template <int R, int DIR>
__device__ __forceinline__ void fft_stage(const float2* __restrict__ src, float2* __restrict__ dst, int n,
                                          int npen, int stride, int ns, const float2* __restrict__ tw) {
  const int nb = n / R;
  const int tot = nb * npen;
  const int twstep = n / (ns * R);
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    const int p = t / nb;
    const int j = t - p * nb;
    const int k = j % ns;
    const float2* sp = src + p * stride;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = sp[j + r * nb];
    if (ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = __ldg(tw + r * k * twstep);
        if (DIR > 0) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    dftR<R, DIR>(v);
    float2* dp = dst + p * stride;
    const int base = (j / ns) * ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dp[base + r * ns] = v[r];
  }
}

// Transforms npen pencils held in a (pencil p at a + p*stride); b is scratch
// of the same shape.  Returns the buffer that holds the result.  Must be
// called by every thread of the block; ends with a __syncthreads().
template <int DIR>
__device__ float2* fft_smem(float2* a, float2* b, int npen, int stride, const FftPlan& P,
                            const float2* __restrict__ tw) {
  int ns = 1;
  for (int s = 0; s < P.nst; ++s) {
    const int R = P.radix[s];
    switch (R) {
      case 8: fft_stage<8, DIR>(a, b, P.n, npen, stride, ns, tw); break;
      case 4: fft_stage<4, DIR>(a, b, P.n, npen, stride, ns, tw); break;
      case 2: fft_stage<2, DIR>(a, b, P.n, npen, stride, ns, tw); break;
      case 5: fft_stage<5, DIR>(a, b, P.n, npen, stride, ns, tw); break;
      default: fft_stage<3, DIR>(a, b, P.n, npen, stride, ns, tw); break;
    }
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
    ns *= R;
  }
  return a;
}

}  // namespace fkp
