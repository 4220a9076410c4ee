// k_noalloc.cu - fkp_power_from_grid_noalloc: the multipole estimator on a
// caller-supplied field for small grids, with every device buffer it needs
// placed in one file-scope device array instead of allocated memory.
//
// Who it is for: callers that may not allocate device memory once they are
// running -- applications that reserve all device memory up front for their
// own pool, latency-critical loops that forbid allocation after start-up, and
// host frameworks that load this library as a plugin without giving it an
// allocator.  cudaMalloc in such a process either fails or stalls the other
// work on the device.
//
// What it shares with the plan-based path: the same kernels (x-, y- and
// z-passes and the bin reduction), launched on buffers carved out of the
// static array.  It takes geometry and bins per call and builds the small
// host tables (twiddles, n^2 -> bin look-up table, window) each time.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "fkp_internal.h"

namespace fkp {
namespace {

constexpr int kNaMaxN = 64;      // largest grid side accepted
constexpr int kNaMaxBins = 64;   // largest number of P bins accepted
constexpr int kNaMaxDevices = 64;

// Byte offsets of the buffers inside the scratch array (256-byte aligned).
constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kNaTilesX = (kNaMaxN / 2 + 1 + 7) / 8;
constexpr size_t kNaField = (size_t)kNaMaxN * kNaTilesX * kNaMaxN * 8;          // complex values per field
constexpr size_t kNaBlkZ = kNaTilesX * kNaMaxN;                                  // z-pass blocks
constexpr size_t kNaN2 = 3 * (kNaMaxN / 2) * (kNaMaxN / 2) + 1;                  // LUT entries
constexpr size_t kOffS1 = 0;
constexpr size_t kOffS2 = kOffS1 + align256(sizeof(float2) * kMaxFields * kNaField);
constexpr size_t kOffTw = kOffS2 + align256(sizeof(float2) * 9 * kNaField);
constexpr size_t kOffLut = kOffTw + align256(sizeof(float2) * kNaMaxN);
constexpr size_t kOffWinv = kOffLut + align256(sizeof(short) * kNaN2);
constexpr size_t kOffPart = kOffWinv + align256(sizeof(float) * 3 * kNaMaxN);
constexpr size_t kOffPartc = kOffPart + align256(sizeof(double) * BQ_N * kNaMaxBins * kNaBlkZ);
constexpr size_t kOffBins = kOffPartc + align256(sizeof(int) * kNaMaxBins * kNaBlkZ);
constexpr size_t kOffBinc = kOffBins + align256(sizeof(double) * BQ_N * kNaMaxBins);
constexpr size_t kOffErr = kOffBinc + align256(sizeof(long long) * kNaMaxBins);
constexpr size_t kNaBytes = kOffErr + 256;  // about 42 MB

}  // namespace

// The scratch array.  Every GPU that loads the library holds it until the
// process exits.  All calls on a device share it: a call clears what must
// start at zero (the error flags) and overwrites the rest, so calls whose
// GPU work overlaps -- on two streams, or from two threads -- race on it.
static __device__ __align__(256) unsigned char g_fkp_noalloc_scratch[kNaBytes];

namespace {

std::mutex g_na_mu;
void* g_na_ptr[kNaMaxDevices] = {};

// The array's device address for the current device.  In host code the
// symbol is only a host-side stand-in, so the address is looked up once per
// device with that device current.
int na_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kNaMaxDevices) return set_error(FKP_EINVAL, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_fkp_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_error(FKP_ECUDA, "cudaGetSymbolAddress for the static scratch failed: %s", cudaGetErrorString(e));
    g_na_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_na_ptr[dev]);
  return FKP_OK;
}

bool na_radix(int n, FftPlan& p) {
  p.n = n;
  p.nst = 0;
  int m = n;
  const int rs[5] = {8, 4, 2, 5, 3};
  for (int r : rs)
    while (m % r == 0) {
      if (p.nst >= 8) return false;
      p.radix[p.nst++] = r;
      m /= r;
    }
  return m == 1;
}

}  // namespace
}  // namespace fkp

using namespace fkp;

#define NCK(call)                                                                                   \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return set_error(FKP_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
  } while (0)

extern "C" int fkp_power_from_grid_noalloc(const fkp_geometry_t* geom, const fkp_pbins_t* pb, const float* F,
                                           double I22, double N0, void* stream, fkp_power_out* out) {
  if (!geom || !pb || !F) return set_error(FKP_EINVAL, "NULL argument");
  const int N = geom->N;
  if (N < 8 || N > kNaMaxN || (N & 1))
    return set_error(FKP_EINVAL, "grid N=%d: this entry point accepts even N <= %d (its static scratch is sized "
                                 "for that); use a plan for larger grids", N, kNaMaxN);
  if (pb->nbins < 1 || pb->nbins > kNaMaxBins || !(pb->dk > 0) || !(pb->kmin >= 0))
    return set_error(FKP_EINVAL, "bad P bins: this entry point accepts 1..%d bins, dk > 0, kmin >= 0", kNaMaxBins);
  if (geom->assign < 2 || geom->assign > 4)
    return set_error(FKP_EINVAL, "assign must be 2 (CIC), 3 (TSC) or 4 (PCS)");
  if (geom->interlace) return set_error(FKP_EINVAL, "a given field has no interlaced partner");
  if (!(geom->L > 0)) return set_error(FKP_EINVAL, "box side L must be positive");
  FftPlan fp;
  if (!na_radix(N, fp)) return set_error(FKP_EINVAL, "grid N=%d is not a product of 2, 3 and 5", N);
  int dev = 0;
  NCK(cudaGetDevice(&dev));
  unsigned char* base = nullptr;
  int rc = na_scratch(dev, &base);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  MomentTable mt;
  build_moments(4, mt);
  if (!moments_match(mt) || !moments_identities_hold(mt, 4))
    return set_error(FKP_ESTATE, "internal: moment table inconsistent");
  GeomDev g{};
  g.N = N;
  g.NH = N / 2 + 1;
  g.H = (float)(geom->L / N);
  g.invH = (float)(N / geom->L);
  g.ox = (float)geom->origin[0];
  g.oy = (float)geom->origin[1];
  g.oz = (float)geom->origin[2];
  g.rx = (float)(geom->origin[0] - geom->observer[0]);
  g.ry = (float)(geom->origin[1] - geom->observer[1]);
  g.rz = (float)(geom->origin[2] - geom->observer[2]);
  g.los_inf = geom->observer_at_infinity ? 1 : 0;
  const double l = std::sqrt(geom->los[0] * geom->los[0] + geom->los[1] * geom->los[1] + geom->los[2] * geom->los[2]);
  if (g.los_inf && !(l > 0)) return set_error(FKP_EINVAL, "los must be nonzero when the observer is at infinity");
  g.lx = l > 0 ? (float)(geom->los[0] / l) : 0.f;
  g.ly = l > 0 ? (float)(geom->los[1] / l) : 0.f;
  g.lz = l > 0 ? (float)(geom->los[2] / l) : 1.f;
  g.assign = geom->assign;
  g.periodic = geom->periodic ? 1 : 0;
  g.P_fkp = (float)geom->P_fkp;
  g.P_fkp_lo = (float)(geom->P_fkp - (double)g.P_fkp);
  g.alpha_mode = geom->alpha_mode;
  observer_node(g);

  // host tables (FP64, rounded once)
  const double kf = 2.0 * M_PI / geom->L;
  const int n2max = 3 * (N / 2) * (N / 2);
  std::vector<short> lut(n2max + 1, -1);
  for (int n2 = 1; n2 <= n2max; ++n2) {
    const double k = kf * std::sqrt((double)n2);
    long b = (long)std::floor((k - pb->kmin) / pb->dk);
    if (b < -1) b = -1;
    if (b > pb->nbins) b = pb->nbins;
    while (b >= 0 && k < pb->kmin + pb->dk * b) --b;
    while (b < pb->nbins && b >= -1 && k >= pb->kmin + pb->dk * (b + 1)) ++b;
    if (b >= 0 && b < pb->nbins) lut[n2] = (short)b;
  }
  std::vector<float2> tw(N);
  for (int m = 0; m < N; ++m) {
    const double a = 2.0 * M_PI * (double)m / (double)N;
    tw[m] = make_float2((float)std::cos(a), (float)-std::sin(a));
  }
  std::vector<float> winv(3 * N, 1.0f);
  if (geom->compensate)
    for (int i = 0; i < N; ++i) {
      const int n = i <= N / 2 ? i : i - N;
      const double t = M_PI * n / N;
      const double sv = n == 0 ? 1.0 : std::sin(t) / t;
      for (int a = 0; a < 3; ++a) winv[a * N + i] = (float)(1.0 / std::pow(sv, geom->assign));
    }

  float2* S1 = reinterpret_cast<float2*>(base + kOffS1);
  float2* S2 = reinterpret_cast<float2*>(base + kOffS2);
  float2* d_tw = reinterpret_cast<float2*>(base + kOffTw);
  short* d_lut = reinterpret_cast<short*>(base + kOffLut);
  float* d_winv = reinterpret_cast<float*>(base + kOffWinv);
  double* d_part = reinterpret_cast<double*>(base + kOffPart);
  int* d_partc = reinterpret_cast<int*>(base + kOffPartc);
  double* d_bins = reinterpret_cast<double*>(base + kOffBins);
  long long* d_binc = reinterpret_cast<long long*>(base + kOffBinc);
  int* d_err = reinterpret_cast<int*>(base + kOffErr);
  NCK(cudaMemcpyAsync(d_tw, tw.data(), sizeof(float2) * N, cudaMemcpyHostToDevice, s));
  NCK(cudaMemcpyAsync(d_lut, lut.data(), sizeof(short) * (n2max + 1), cudaMemcpyHostToDevice, s));
  NCK(cudaMemcpyAsync(d_winv, winv.data(), sizeof(float) * 3 * N, cudaMemcpyHostToDevice, s));
  NCK(cudaMemsetAsync(d_err, 0, sizeof(int) * 4, s));

  int dsm = 1;
  NCK(cudaDeviceGetAttribute(&dsm, cudaDevAttrMultiProcessorCount, dev));
  NCK(launch_xpass(nullptr, F, g, mt, fp, d_tw, S1, dsm, s));
  NCK(launch_ypass(S1, nullptr, F, g, mt, fp, d_tw, S2, d_err + 1, s));
  ZParams zp;
  zp.nbins = pb->nbins;
  zp.lmax = 4;
  zp.kf = (float)kf;
  zp.lut = d_lut;
  zp.winv = d_winv;
  zp.mode = 0;
  zp.nshells = 0;
  zp.nsh2 = 0;
  zp.slut = nullptr;
  zp.E = nullptr;
  zp.mm = 0;
  zp.split68 = 1;
  NCK(launch_zpass(S2, g, mt, fp, d_tw, zp, d_part, d_partc, d_err + 1, s, dsm, z_threads_for(N)));
  NCK(launch_reduce_bins(d_part, d_partc, zpass_blocks(N, z_threads_for(N), dsm), pb->nbins, d_bins, d_binc, s));

  const int nb = pb->nbins;
  std::vector<double> hb(BQ_N * nb);
  std::vector<long long> hc(nb);
  int herr[2] = {0, 0};
  NCK(cudaMemcpyAsync(hb.data(), d_bins, sizeof(double) * BQ_N * nb, cudaMemcpyDeviceToHost, s));
  NCK(cudaMemcpyAsync(hc.data(), d_binc, sizeof(long long) * nb, cudaMemcpyDeviceToHost, s));
  NCK(cudaMemcpyAsync(herr, d_err, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
  NCK(cudaStreamSynchronize(s));
  if (herr[1] != 0)
    return set_error(FKP_ETIMEOUT, "a bounded device-side wait for a tile copy gave up (flags 0x%x)", herr[1]);
  if (!out) return FKP_OK;
  out->alpha = 0; out->I22 = I22; out->I33 = 0; out->N0 = N0; out->N0_fkp = 0; out->S3 = 0;
  out->W_g = out->W_r = 0; out->n_gal = out->n_ran = 0;
  for (int a = 0; a < 6; ++a) out->Lab[a] = 0;
  for (int i = 0; i < 8; ++i) out->timing_ms[i] = 0.f;
  out->graph = 0;
  for (int b = 0; b < nb; ++b) {
    const double n = (double)hc[b];
    const double s00 = hb[BQ_F00 * nb + b], s20 = hb[BQ_F20 * nb + b], s40 = hb[BQ_F40 * nb + b],
                 s22 = hb[BQ_F22 * nb + b], sk = hb[BQ_K * nb + b];
    const double nan = std::nan("");
    if (out->nmodes) out->nmodes[b] = hc[b];
    if (out->k_eff) out->k_eff[b] = n > 0 ? sk / n : nan;
    if (out->mono_raw) out->mono_raw[b] = n > 0 ? s00 / n / I22 : nan;
    if (out->P0) out->P0[b] = n > 0 ? (s00 / n - N0) / I22 : nan;
    if (out->P2) out->P2[b] = n > 0 ? 5.0 * s20 / n / I22 : nan;
    if (out->P4) out->P4[b] = n > 0 ? 9.0 * s40 / n / I22 : nan;
    if (out->P4b) out->P4b[b] = n > 0 ? (17.5 * s22 - 5.0 * s20 - 3.5 * s00) / n / I22 : nan;
    // split l = 6, 8 (Sec. II.B after eq. P4fast): L_2 L_4 and L_4^2 in Legendre polynomials
    const double s42 = hb[BQ_F42 * nb + b], s44 = hb[BQ_F44 * nb + b];
    const double s60 = 11.0 / 5.0 * (s42 - 2.0 / 7.0 * s20 - 20.0 / 77.0 * s40);
    const double s80 = 1287.0 / 490.0 * (s44 - s00 / 9.0 - 100.0 / 693.0 * s20 - 162.0 / 1001.0 * s40 - 20.0 / 99.0 * s60);
    if (out->P6b) out->P6b[b] = n > 0 && true ? 13.0 * s60 / n / I22 : nan;
    if (out->P8b) out->P8b[b] = n > 0 && true ? 17.0 * s80 / n / I22 : nan;
  }
  return FKP_OK;
}
