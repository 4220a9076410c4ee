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
  double P_fkp_d;      // P_FKP in FP64 (the scalar sums)
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
enum { BQ_K = 0, BQ_F00, BQ_F20, BQ_F40, BQ_F22, BQ_N };
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

// The same weight in FP64 for the scalar sums (alpha, I_22, N_0, I_33, S_3):
// the FP32 reciprocal of d = 1 + nbar P_FKP refined by one Newton-Raphson
// step r1 = r0 + r0 (1 - d r0), which squares its relative error (2^-24 ->
// about 1e-14).  Weights given with the catalog are taken as they are.
__device__ __forceinline__ double fkp_weight_f64(const CatDev& c, long long i, double Pfkp) {
  if (c.w) return (double)__ldg(c.w + i);
  const double d = fma((double)__ldg(c.nbar + i), Pfkp, 1.0);
  const double r0 = (double)__frcp_rn((float)d);
  return fma(r0, fma(-d, r0, 1.0), r0);
}

}  // namespace fkp
