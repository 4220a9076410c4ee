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

// ----------------------------------------------------------------------------
// Compile-time-sized FFT on interleaved pencils.
//
// P pencils of length N are interleaved in shared memory: element i of pencil
// p sits at buf[i * P + p], so the tile of P consecutive k_x columns that a
// pass reads from global memory is already in FFT layout.  N, P, the block
// size and the radix sequence are template constants, so every index
// division is by a constant and every loop unrolls.  Twiddles come from a
// shared-memory table.
// ----------------------------------------------------------------------------

namespace fkp {

__host__ __device__ constexpr int radix_count(int n) {
  int c = 0;
  while (n % 8 == 0) { n /= 8; ++c; }
  while (n % 4 == 0) { n /= 4; ++c; }
  while (n % 2 == 0) { n /= 2; ++c; }
  while (n % 5 == 0) { n /= 5; ++c; }
  while (n % 3 == 0) { n /= 3; ++c; }
  return c;
}

__host__ __device__ constexpr int radix_at(int n, int s) {
  int i = 0;
  while (n % 8 == 0) { if (i == s) return 8; n /= 8; ++i; }
  while (n % 4 == 0) { if (i == s) return 4; n /= 4; ++i; }
  while (n % 2 == 0) { if (i == s) return 2; n /= 2; ++i; }
  while (n % 5 == 0) { if (i == s) return 5; n /= 5; ++i; }
  while (n % 3 == 0) { if (i == s) return 3; n /= 3; ++i; }
  return 1;
}

// Shared-memory index of element i of pencil p among P interleaved pencils.
// With SWZ (P a power of two) the pencil slot is XOR-swizzled by i >> 1:
// one pencil read or written at consecutive i, and all pencils at one i,
// then both fall in distinct banks (per half-warp).
template <int P, bool SWZ>
__device__ __forceinline__ int ilv(int i, int p) {
  if constexpr (SWZ) {
    static_assert((P & (P - 1)) == 0, "swizzled interleave needs a power-of-two pencil count");
    return i * P + (p ^ ((i >> 1) & (P - 1)));
  } else {
    return i * P + p;
  }
}

// Row permutation of the interleaved layout with P = 8 pencils (a row is
// the 8 values of one index i, 64 bytes, half of the shared-memory banks):
// rows i and i ^ 1 swap when bit 3 of i is set.  A first radix-8 stage writes
// rows 8j + r for four consecutive j per warp, all of one parity, i.e. all
// into the same half of the banks (two wavefronts too many); with the
// permutation consecutive j alternate halves, while runs of four
// consecutive rows (every other access of the stages) stay spread over both.
__host__ __device__ __forceinline__ constexpr int rowx(int i) { return i ^ ((i >> 3) & 1); }

// Shared-memory index of element i of pencil p in the row-permuted layout.
template <int P, bool SWZ, bool RX>
__device__ __forceinline__ int ilvx(int i, int p) {
  if constexpr (RX) return rowx(i) * P + p;
  else return ilv<P, SWZ>(i, p);
}

// The block is 2-D: threadIdx.x = pencil (blockDim.x == P), threadIdx.y
// strides over the N/R butterflies of a stage (blockDim.y == NT / P).
// RXI / RXO: the stage reads / writes the row-permuted layout.
template <int N, int P, int NT, int DIR, int R, int NS, bool SWZ, bool RXI = false, bool RXO = false>
__device__ __forceinline__ void fft_ct_stage(const float2* __restrict__ src, float2* __restrict__ dst,
                                             const float2* __restrict__ tw) {
  constexpr int NB = N / R;
  constexpr int JT = NT / P;
  constexpr int TWS = N / (NS * R);
  const int p = threadIdx.x;
#pragma unroll
  for (int j0 = 0; j0 < NB; j0 += JT) {
    const int j = j0 + (int)threadIdx.y;
    if ((NB % JT) == 0 || j < NB) {
      const int k = j % NS;
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = src[ilvx<P, SWZ, RXI>(j + r * NB, p)];
      if (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[r * k * TWS];
          if (DIR > 0) w.y = -w.y;
          v[r] = cmul(v[r], w);
        }
      }
      dftR<R, DIR>(v);
      const int base = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[ilvx<P, SWZ, RXO>(base + r * NS, p)] = v[r];
    }
  }
}

template <int N, int P, int NT, int DIR, int S, int NS, bool SWZ, bool RX = false>
__device__ __forceinline__ float2* fft_ct_run(float2* a, float2* b, const float2* tw) {
  if constexpr (S == radix_count(N)) {
    return a;
  } else {
    constexpr int R = radix_at(N, S);
    fft_ct_stage<N, P, NT, DIR, R, NS, SWZ, (RX && (S > 0)), RX>(a, b, tw);
    __syncthreads();
    return fft_ct_run<N, P, NT, DIR, S + 1, NS * R, SWZ, RX>(b, a, tw);
  }
}

// Transforms P interleaved pencils held in a (b is scratch of the same size).
// Returns the buffer holding the result.  All NT threads of the (P, NT/P)
// block call it; it ends with a __syncthreads().  RX (P = 8, no swizzle):
// the input is in the natural interleave and the result in the
// row-permuted one (element i of pencil p at rowx(i) * 8 + p).
template <int N, int P, int NT, int DIR, bool SWZ = false, bool RX = false>
__device__ __forceinline__ float2* fft_ct(float2* a, float2* b, const float2* tw) {
  static_assert(!RX || (P == 8 && !SWZ), "the row permutation is for 8 unswizzled pencils");
  return fft_ct_run<N, P, NT, DIR, 0, 1, SWZ, RX>(a, b, tw);
}

// Stages S .. SEND-1 of fft_ct_run; returns the buffer holding their result.
template <int N, int P, int NT, int DIR, int S, int NS, int SEND, bool SWZ, bool RX>
__device__ __forceinline__ float2* fft_ct_upto(float2* a, float2* b, const float2* tw) {
  if constexpr (S == SEND) {
    return a;
  } else {
    constexpr int R = radix_at(N, S);
    fft_ct_stage<N, P, NT, DIR, R, NS, SWZ, (RX && (S > 0)), RX>(a, b, tw);
    __syncthreads();
    return fft_ct_upto<N, P, NT, DIR, S + 1, NS * R, SEND, SWZ, RX>(b, a, tw);
  }
}

__host__ __device__ constexpr int radix_prod(int n, int s) {
  int p = 1;
  for (int i = 0; i < s; ++i) p *= radix_at(n, i);
  return p;
}

// Whether fft_ct_fused applies: the last stage's butterflies per pencil (N/R)
// come in whole rounds of the NT/P threads of a pencil.
template <int N, int P, int NT>
__host__ __device__ constexpr bool fft_fusable() {
  return N > 0 && radix_count(N) >= 2 && (N / radix_at(N, radix_count(N) - 1)) % (NT / P) == 0;
}

// The transform of fft_ct<N, P, NT, DIR, SWZ, RX> whose last stage hands its
// outputs to the caller instead of storing them: thread (p, y) receives
// output index y + i NT/P of pencil p as f(i, value), for every i in
// [0, N P / NT), each exactly once, in registers.  The earlier stages run as
// in fft_ct and end with a __syncthreads(); the last one reads the buffer
// returned in *last_src and stores nothing, so the other buffer is free and
// the caller synchronises before either is reused.
template <int N, int P, int NT, int DIR, bool SWZ, bool RX, class F>
__device__ __forceinline__ void fft_ct_fused(float2* a, float2* b, const float2* tw, F&& f,
                                             const float2** last_src = nullptr) {
  static_assert(fft_fusable<N, P, NT>(), "the last stage's outputs do not map onto the threads' runs");
  constexpr int SL = radix_count(N) - 1;
  constexpr int R = radix_at(N, SL);
  constexpr int NS = radix_prod(N, SL);  // = N / R
  constexpr int NB = N / R;
  constexpr int JT = NT / P;
  const float2* src = fft_ct_upto<N, P, NT, DIR, 0, 1, SL, SWZ, RX>(a, b, tw);
  if (last_src) *last_src = src;
  const int p = threadIdx.x;
#pragma unroll
  for (int j0 = 0; j0 < NB; j0 += JT) {
    // last stage: k = j mod NS = j, outputs j + r NS
    const int j = j0 + (int)threadIdx.y;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[ilvx<P, SWZ, RX>(j + r * NB, p)];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 w = tw[r * j * (N / (NS * R))];
      if (DIR > 0) w.y = -w.y;
      v[r] = cmul(v[r], w);
    }
    dftR<R, DIR>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) f((j0 + r * NS) / JT, v[r]);
  }
}

// Runtime-N version on the same interleaved layout (sizes without a
// compiled specialisation).
template <int R, int DIR, bool SWZ>
__device__ __forceinline__ void fft_rt_stage(const float2* __restrict__ src, float2* __restrict__ dst, int n, int P,
                                             int ns, const float2* __restrict__ tw) {
  const int nb = n / R;
  const int tot = nb * P;
  const int tws = n / (ns * R);
  const int nthr = blockDim.x * blockDim.y;
  for (int t = threadIdx.y * blockDim.x + threadIdx.x; t < tot; t += nthr) {
    const int p = t % P;
    const int j = t / P;
    const int k = j % ns;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[SWZ ? (j + r * nb) * P + (p ^ (((j + r * nb) >> 1) & (P - 1))) : (j + r * nb) * P + p];
    if (ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = tw[r * k * tws];
        if (DIR > 0) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    dftR<R, DIR>(v);
    const int base = (j / ns) * ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = base + r * ns;
      dst[SWZ ? i * P + (p ^ ((i >> 1) & (P - 1))) : i * P + p] = v[r];
    }
  }
}

template <int DIR, bool SWZ = false>
__device__ float2* fft_rt(float2* a, float2* b, int P, const FftPlan& fp, const float2* tw) {
  int ns = 1;
  for (int s = 0; s < fp.nst; ++s) {
    const int R = fp.radix[s];
    switch (R) {
      case 8: fft_rt_stage<8, DIR, SWZ>(a, b, fp.n, P, ns, tw); break;
      case 4: fft_rt_stage<4, DIR, SWZ>(a, b, fp.n, P, ns, tw); break;
      case 2: fft_rt_stage<2, DIR, SWZ>(a, b, fp.n, P, ns, tw); break;
      case 5: fft_rt_stage<5, DIR, SWZ>(a, b, fp.n, P, ns, tw); break;
      default: fft_rt_stage<3, DIR, SWZ>(a, b, fp.n, P, ns, tw); break;
    }
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
    ns *= R;
  }
  return a;
}

// N = 0 selects the runtime version.  SWZ: swizzled interleave (see ilv).
// RX: the compile-time version leaves its result row-permuted (see fft_ct);
// the runtime version ignores it, so read results through res_row<N, RX>.
template <int N, int P, int NT, int DIR, bool SWZ = false, bool RX = false>
__device__ __forceinline__ float2* fft_any(float2* a, float2* b, const FftPlan& fp, const float2* tw) {
  if constexpr (N > 0) return fft_ct<N, P, NT, DIR, SWZ, RX>(a, b, tw);
  else return fft_rt<DIR, SWZ>(a, b, P, fp, tw);
}

// Row of index i in the result of fft_any<N, ..., RX>.
template <int N, bool RX>
__device__ __forceinline__ int res_row(int i) {
  if constexpr (N > 0 && RX) return rowx(i);
  else return i;
}

// ----------------------------------------------------------------------------
// Bulk (TMA) copies of contiguous tiles into shared memory, completed on an
// mbarrier.  Waits are bounded: after kWaitLimit polls the waiter records an
// error flag and gives up (the host then reports FKP_ETIMEOUT).
// ----------------------------------------------------------------------------

constexpr unsigned kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// 1-D bulk copy global -> shared (addresses 16-byte aligned, size multiple of 16).
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on phase `parity`: at most `limit` polls; returns false (and
// sets *err |= flag) when it gives up.
__device__ __forceinline__ bool mbar_wait_n(uint64_t* bar, uint32_t parity, int* err, int flag, unsigned limit) {
  for (unsigned it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  if (err) atomicOr(err, flag);
  return false;
}

// The passes' wait: kWaitLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int flag) {
  return mbar_wait_n(bar, parity, err, flag, kWaitLimit);
}

}  // namespace fkp
