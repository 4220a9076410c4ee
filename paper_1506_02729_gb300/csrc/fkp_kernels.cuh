// fkp_kernels.cuh - parameter blocks and launch wrappers shared by the
// kernel translation units and the C-ABI host code.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fkp_fft.cuh"

namespace fkp {

constexpr int kMaxFields = 16;   // 1 + 5 + 10 trace-reduced moment fields per base grid
constexpr int kMaxGroups = 9;    // k_z-power groups per base grid
constexpr int kMaxSweeps = 6;    // y-pass sweeps (fields read in turn into up to two groups)
constexpr int kMaxMembers = 5;   // fields per sweep
constexpr int kMaxBins = 512;    // P bins
constexpr int kMaxShells = 64;   // bispectrum shells
constexpr double kFixScale = 1099511627776.0;       // 2^40: fixed-point scale of the grids
constexpr float kFixScaleF = 1099511627776.0f;
constexpr float kFixInvF = 9.094947017729282379e-13f;  // 2^-40

// Geometry as the kernels see it.
struct GeomDev {
  int N, NH;           // grid side, N/2 + 1
  float H, invH;       // cell size and its inverse
  float ox, oy, oz;    // origin (box corner)
  float rx, ry, rz;    // node 0 relative to the observer: origin - observer
  int los_inf;         // observer at infinity
  float lx, ly, lz;    // unit line of sight when los_inf
  int assign;          // 2 CIC, 3 TSC
  int periodic;
  float P_fkp;
  int alpha_mode;
  float P_fkp_lo;      // P_FKP - P_fkp (the scalar sums carry P_FKP as a float pair)
  int obs_x, obs_y, obs_z;  // grid node at the observer (x^ = 0 there), or -1
};

// Moment fields of one base grid: field q is grid * xh_x^e[q][0] xh_y^e[q][1]
// xh_z^e[q][2].  The y-pass reads the fields sweep by sweep; sweep s reads
// s_field[s][0..s_nmem) and accumulates s_nout <= 2 output groups
// s_out[s][o], member m entering output o with the coefficient
// sum_t s_c[s][m][o][t] nx^s_i[s][m][o][t] ny^s_j[s][m][o][t] (t < 2), and the
// output s_obs[s] (if >= 0) receiving the observer node's F.  The z-pass then
// adds group g to F_0 (g_f0), g_c2 nz^g_p2 times it to S_2 and g_c4 nz^g_p4
// times it to S_4.
struct MomentTable {
  int nfields, ngroups, nsweeps;
  unsigned char e[kMaxFields][3];
  int s_nmem[kMaxSweeps], s_nout[kMaxSweeps], s_out[kMaxSweeps][2], s_obs[kMaxSweeps];
  int s_field[kMaxSweeps][kMaxMembers];
  float s_c[kMaxSweeps][kMaxMembers][2][2];
  unsigned char s_i[kMaxSweeps][kMaxMembers][2][2];
  unsigned char s_j[kMaxSweeps][kMaxMembers][2][2];
  int g_f0[kMaxGroups];
  float g_c2[kMaxGroups], g_c4[kMaxGroups];
  unsigned char g_p2[kMaxGroups], g_p4[kMaxGroups];
};

// Number of per-block FP64 partial sums the scalar kernels produce.
// gal: n, sum w, sum w^2, sum w^3 ; ran: n, sum w, sum w^2, sum w^3, sum nbar w^2, sum nbar^2 w^3
enum { SC_G_W = 0, SC_G_W2, SC_G_W3, SC_R_W, SC_R_W2, SC_R_W3, SC_R_NW2, SC_R_N2W3, SC_NSUM };
// L^ab partial sums (randoms): sum w xh_a xh_b, order xx yy zz xy yz zx
enum { LAB_NSUM = 6 };
// Device scalars written by the finalize kernel (FP64).
enum { DS_ALPHA = 0, DS_I22, DS_I33, DS_N0, DS_N0FKP, DS_S3, DS_WG, DS_WR, DS_NG, DS_NR, DS_COUNT };
// Per-bin quantities accumulated by the z-pass.
enum { BQ_K = 0, BQ_F00, BQ_F20, BQ_F40, BQ_F22, BQ_F42, BQ_F44, BQ_N };
// Per-shell quantities of the F^w pass (same slots): Re F_0 F^w_0*, Re F_2 F^w_0*,
// Re F_4 F^w_0*, Re F_0 F^w_2*, Re F_0 F^w_4*.
enum { SQ_00 = 0, SQ_20, SQ_40, SQ_02, SQ_04 };

// z-pass parameters.
// Several mocks of one plan in one launch of an FFT pass: blockIdx.z picks the
// mock, whose buffers lie at fixed element strides from the first mock's.
// n = 1 (strides unused) is the single-mock launch.
struct MockBatch {
  int n = 1;
  long long in = 0;    // stride of the pass's input (x: grid; y: S1; z: S2)
  long long in2 = 0;   // y: stride of the grid (observer-node value)
  long long out = 0;   // stride of the output (x: S1; y: S2; z: partial bin sums)
  long long out2 = 0;  // z: stride of the partial bin counts
};

struct ZParams {
  int nbins;
  int lmax;          // 0, 2 or 4
  float kf;          // 2 pi / L
  const short* lut;  // n^2 -> bin or -1
  const float* winv; // [3][N]: 1/sinc^p per axis index (ones when not compensating)
  int mode;          // 0 P bins, 1 P bins + export, 2 F^w shell sums
  int nshells;
  int nsh2;          // slut covers n^2 < nsh2
  const signed char* slut;  // n^2 -> shell or -1
  float2* E;         // [3][2mm+1][2mm+1][mm+1]: F_0, F_2, F_4 on the shells
  int mm;            // largest |n_a| inside the outermost shell
  // interlaced pair of grids: groups [ngroups, 2 ngroups) come from the
  // second grid (nodes half a cell further); hph[i] = e^{-i pi n/N} with n the
  // signed index of i: the z-pass multiplies those groups after its FFT by
  // hph[k_x] hph[k_y] hph[k_z]; scale = 1/2 averages the two grids (1 without
  // interlacing)
  int interlace = 0;
  const float2* hph = nullptr;
  float scale = 1.f;
  int split68 = 0;   // accumulate Re F_4 F_2* and |F_4|^2 (P_6b, P_8b)
};

// Catalog on the device.
struct CatDev {
  const float *x, *y, *z, *w, *nbar;
  long long n;
};

// Compensated FP32 accumulator (per-thread partial sums; the block and grid
// levels sum in FP64).
struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Block-wide FP64 sum of one value per thread; the result is valid in thread 0.
__device__ __forceinline__ double block_sum_f64(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) r += sh[i];
  }
  return r;
}

// FKP weight w = 1/(1 + nbar P_FKP) unless the catalog carries weights.
__device__ __forceinline__ float fkp_weight(const CatDev& c, long long i, float Pfkp) {
  return c.w ? __ldg(c.w + i) : 1.0f / (1.0f + __ldg(c.nbar + i) * Pfkp);
}

// Double-single ("float-float") arithmetic for the scalar sums: a value is an
// unevaluated pair hi + lo of FP32 numbers (about 48 significant bits), with
// Knuth's TwoSum for exact additions and the FMA-based TwoProduct for exact
// products.  It gives the FP64-level accuracy the normalisation and shot-noise
// sums need at FP32 throughput (FP64 units are few on this part).
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = a.hi * b.hi;
  return {p, fmaf(a.hi, b.hi, -p) + (a.hi * b.lo + a.lo * b.hi)};
}
__device__ __forceinline__ FF ff_mul(FF a, float b) {
  const float p = a.hi * b;
  return {p, fmaf(a.hi, b, -p) + a.lo * b};
}
// Running sum of float pairs.
struct FFSum {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(FF x) {
    const FF s = ff_two_sum(hi, x.hi);
    hi = s.hi;
    lo += s.lo + x.lo;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// The FKP weight as a float pair for the scalar sums: d = 1 + nbar P_FKP
// exactly as a pair, the FP32 reciprocal r0 of its leading part, and one
// Newton-Raphson step w = r0 + r0 (1 - d r0) with the residual formed by FMA
// (relative error about 2^-46).  Weights given with the catalog are exact.
__device__ __forceinline__ FF fkp_weight_ff(const CatDev& c, long long i, float Ph, float Pl) {
  if (c.w) return {__ldg(c.w + i), 0.f};
  const float nb = __ldg(c.nbar + i);
  const float p = nb * Ph;
  const float pe = fmaf(nb, Ph, -p) + nb * Pl;  // nbar P = p + pe
  const FF d = ff_two_sum(1.f, p);               // 1 + p = d.hi + d.lo
  const float dl = d.lo + pe;
  const float r0 = __frcp_rn(d.hi);
  const float res = fmaf(-dl, r0, fmaf(-d.hi, r0, 1.f));
  return ff_two_sum(r0, r0 * res);
}

}  // namespace fkp
