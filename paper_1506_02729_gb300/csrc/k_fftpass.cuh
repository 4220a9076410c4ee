// k_fftpass.cuh - the three FFT passes of the power-spectrum path: shared
// helpers (the x-pass is in k_xpass.cu, the y-pass in k_ypass.cu, the z-pass
// in k_zpass.cu).
//
//   x-pass  per grid row (blocks walk rows, the next row's values loaded
//           while this one is transformed): moment fields F x^_a x^_b (...)
//           built at the nodes about the observer (eqs. Qij, Qijkl, Qab), two
//           real fields packed per complex pencil (XOR-swizzled interleave),
//           FFT along x, unpacked into half spectra.
//   y-pass  per (z, k_x tile): FFT of each field along y, then the k_x, k_y
//           polynomials of eqs. delta2b and delta4b (with the multinomial
//           multiplicities and the trace identities of the unit vector x^),
//           summed into k_z-power groups.
//   z-pass  per (k_y, k_x tile), persistent blocks walking their tiles with
//           the next tile's first copy in flight: FFT of each group along z, Legendre
//           recombination F_2 = 3/2 S_2/|n|^2 - F_0/2 and
//           F_4 = 35/8 S_4/|n|^4 - 5/2 F_2 - 7/8 F_0 (eqs. F2, delta4),
//           window compensation and shell binning (eq. shell).
//
// The x-pass grid and the y-pass block shape are chosen per grid by timing
// when a plan is made (PassSchedule); the z-pass block shape is fixed per
// grid (it sets how the bin sums are split into FP32 runs).  Layouts are tile-major so that every tile a pass
// reads is one contiguous block, fetched with a bulk (TMA) copy while the
// previous one is being transformed:
//   S1[field][z][xt][y][c]   (k_x = 8 xt + c), written by the x-pass
//   S2[group][xt][ky][z][c]  written by the y-pass, read by the z-pass
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fkp_internal.h"

namespace fkp {

constexpr int kT = 8;        // k_x columns per tile (64 bytes of complex64)
// y-pass blocks (8, 32), two per SM; z-pass blocks (8, 64), one per SM (its
// three accumulators per point need the registers)
// The y- and z-pass blocks are (8, NT / 8): NT / 8 threads per column, each
// holding RL = 512 / (NT / 8) points (N <= 512).  NT is 256 or 512.
template <int NT>
struct PassShape {
  static constexpr int kRun = NT / kT;
  static constexpr int kRL = (512 + kRun - 1) / kRun;
  static constexpr int kMinBlocks = NT <= 256 ? 2 : 1;
};

__device__ __forceinline__ int smode(int k, int N) { return k <= N / 2 ? k : k - N; }

__device__ __forceinline__ float powi(float v, int e) {
  float r = 1.f;
  for (int i = 0; i < e; ++i) r *= v;
  return r;
}

__device__ __forceinline__ float pw5(const float* h, int e) {
  return e == 0 ? 1.f : (e == 1 ? h[1] : (e == 2 ? h[2] : (e == 3 ? h[3] : h[4])));
}

// Moment-field exponents (i, j, k) of x^_x^i x^_y^j x^_z^k in the order the
// host's moment table uses: F_0; for ell = 2, 4 the components with z power
// p = 0, 1 (j ascending); then zzzz (the trace-reduced set: 1 + 5 + 10).
__host__ __device__ constexpr int nfields_of(int lmax) { return lmax >= 4 ? 16 : (lmax >= 2 ? 6 : 1); }
__host__ __device__ constexpr int field_exp(int q, int a) {
  int idx = 0;
  for (int ell = 0; ell <= 4; ell += 2) {
    for (int p = 0; p <= (ell ? 1 : 0); ++p)
      for (int j = 0; j <= ell - p; ++j) {
        if (idx == q) return a == 0 ? ell - p - j : (a == 1 ? j : p);
        ++idx;
      }
    if (ell == 4 && idx == q) return a == 2 ? 4 : 0;
  }
  return 0;
}

// ----------------------------------------------------------------------------
// k_z-power groups as the z-pass applies them (the host's moment table lists
// the same values; moments_match checks them): group g adds to F_0 (zg_f0),
// zg_c2 nz^zg_p2 times itself to S_2 and zg_c4 nz^zg_p4 times itself to S_4.
// ----------------------------------------------------------------------------

__host__ __device__ constexpr int zg_f0(int g) { return g == 0 ? 1 : 0; }
__host__ __device__ constexpr float zg_c2(int g) {
  return g == 0 ? 1.f : (g == 1 ? 1.f : (g == 2 ? -1.f : (g == 3 ? 1.f : 0.f)));
}
__host__ __device__ constexpr int zg_p2(int g) { return g == 0 ? 2 : (g == 2 ? 2 : (g == 3 ? 1 : 0)); }
__host__ __device__ constexpr float zg_c4(int g) {
  return g == 1 ? 6.f : (g == 3 ? 2.f : (g == 4 || g == 6 || g == 8 ? 1.f : (g == 5 || g == 7 ? -1.f : 0.f)));
}
__host__ __device__ constexpr int zg_p4(int g) {
  return g == 1 || g == 5 ? 2 : (g == 3 || g == 7 ? 3 : (g == 6 ? 1 : (g == 8 ? 4 : 0)));
}

// v^e for e in 0..4 from v and v^2, by selection (no loop).
__device__ __forceinline__ float pwsel(float v, float v2, int e) {
  return e == 0 ? 1.f : (e == 1 ? v : (e == 2 ? v2 : (e == 3 ? v2 * v : v2 * v2)));
}

inline size_t ysm(int N) { return 128 + sizeof(float2) * (3 * (size_t)N * kT + N); }

}  // namespace fkp
