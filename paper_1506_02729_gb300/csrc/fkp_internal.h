// fkp_internal.h - host-side structures of the library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/fkp.h"
#include "fkp_kernels.cuh"

namespace fkp {

// Launch schedule of the FFT passes, chosen per (grid, multipole order) by
// timing the candidates when the first plan of that kind is made.
struct PassSchedule {
  int x_mult = 2;       // x-pass blocks per SM = resident blocks x x_mult (1, 2, 4 or 8)
  int y_threads = 256;  // y-pass block: 256 (two per SM) or 512
  int z_threads = 512;  // z-pass block: 256 or 512 (fixed per grid by z_threads_for, not tuned)
  float ms[3] = {0, 0, 0};  // the chosen x, y, z times when tuned (ms)
  bool tuned = false;
};

struct Context {
  int device = 0;
  size_t budget = 0;
  int nsm = 1;
  std::mutex tune_mu;
  std::map<std::pair<int, int>, PassSchedule> schedules;  // (N, lmax) -> schedule
};

struct Plan {
  Context* ctx = nullptr;
  fkp_geometry_t geom{};
  fkp_pbins_t pb{};
  fkp_bshells_t bs{};
  uint32_t want = 0;
  bool wantB = false;
  // moments with each object's x^ (FKP_XHAT_OBJECT): d_grid then holds the
  // mt.nfields moment grids one after the other (field 0 = F)
  bool per_object = false;
  int lmax = 0;
  MomentTable mt{};
  PassSchedule sched{};
  FftPlan fp{};
  GeomDev g{};
  double min_edge_gap = 0;
  int nblk_cat = 0;
  int nblk_z = 0;  // capacity (in blocks) of the z-pass partial bins: one per tile; the
                   // persistent z-pass writes zpass_blocks(...) <= nblk_z of them

  // power workspace
  unsigned long long *d_grid = nullptr, *d_gridw = nullptr;
  float2 *d_S1 = nullptr, *d_S2 = nullptr, *d_tw = nullptr;
  short* d_lut = nullptr;
  float* d_winv = nullptr;
  double *d_scpart = nullptr, *d_labpart = nullptr, *d_ds = nullptr;
  int* d_err = nullptr;
  // tile binning of the catalogs (gridding)
  int ntiles = 0;
  int *d_tcnt = nullptr, *d_toff = nullptr, *d_titem = nullptr;
  int* d_bhist = nullptr;  // per-block tile counts of the count launches (2 nsm rows)
  float4* d_xyzv = nullptr;
  float* d_vw2 = nullptr;
  size_t sort_cap = 0;
  double* d_zpart = nullptr;
  int* d_zpartc = nullptr;
  double* d_bins = nullptr;
  long long* d_binc = nullptr;

  // bispectrum workspace and tables
  int ntri = 0;
  void* bisp = nullptr;

  // interlaced pair of grids (geom.interlace): the second grid's geometry
  // (nodes half a cell further), its grids, and the half-cell phase table
  // e^{-i pi n/N} by signed index
  bool interlace = false;
  GeomDev g2{};
  unsigned long long *d_grid2 = nullptr, *d_gridw2 = nullptr;
  float2* d_hph = nullptr;
  unsigned long long *rc_grid2 = nullptr, *rc_gridw2 = nullptr;

  // cached random catalog (fkp_plan_cache_randoms): its grids without alpha,
  // R = sum_r w W and R^w = sum_r w^2 W, the per-block partial scalar sums
  // of its count launch, its L^ab sums and its size
  bool rc_valid = false;
  unsigned long long *rc_grid = nullptr, *rc_gridw = nullptr;
  double *rc_part = nullptr, *rc_lab = nullptr;
  int rc_nblk = 0;
  long long rc_n = 0;

  // host catalogs staged on the device (slot 0 galaxies, 1 randoms)
  void* staging[2] = {nullptr, nullptr};
  size_t staging_bytes[2] = {0, 0};
  void* h_pinned = nullptr;
  cudaEvent_t ev[12] = {};
  // the grids' zeroing runs on a side stream beside the count launches
  // (fork and join events, no timing)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  // CUDA graph of the device-catalog power path (gridding, FFT passes,
  // binning), keyed by the catalogs it was captured with
  bool graphs = true;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  CatDev graph_key[2] = {};
  CatDev last_key[2] = {};
  bool last_valid = false;
  int graph_launches = 0;

  // fused multi-mock power (fkp_power_batch): one allocation holding, for up
  // to batch_cap mocks, the grids, pass buffers, partial and final bins,
  // scalars and flags, each mock's at a fixed stride from the first's
  int batch_cap = 0;
  void* batch_mem = nullptr;
  size_t batch_bytes = 0;
  unsigned long long* b_grid = nullptr;
  float2 *b_S1 = nullptr, *b_S2 = nullptr;
  double *b_zpart = nullptr, *b_bins = nullptr, *b_ds = nullptr;
  int *b_zpartc = nullptr, *b_err = nullptr;
  long long* b_binc = nullptr;

  std::vector<void*> buffers;
  size_t bytes_total = 0;
  void* alloc(size_t bytes);
  ~Plan();
};

int set_error(int code, const char* fmt, ...);
// Raises a kernel's dynamic shared-memory limit on the current device to at
// least `bytes`.  The limit is process-wide per kernel and is never lowered
// here, so a launch with a smaller need on another thread stays valid.
cudaError_t raise_smem_limit(const void* func, size_t bytes);
void build_moments(int lmax, MomentTable& mt);
int z_threads_for(int N);
bool moments_identities_hold(const MomentTable& mt, int lmax);
void observer_node(GeomDev& g);
int stage_catalog(Plan* P, const fkp_catalog_t* c, int slot, CatDev& out, cudaStream_t s);
int randoms_of(Plan* P, const fkp_catalog_t* ran, CatDev& r, cudaStream_t s);
int enqueue_grids(Plan* P, const CatDev& gal, const CatDev& ran, cudaStream_t s);
int enqueue_fft_bin(Plan* P, const unsigned long long* gq, const float* gf, cudaStream_t s);
// x- and y-passes of a field into the plan's S2: of the fixed-point grid gq
// (and, interlaced, of gq2 on the second grid) or of the FP32 field gf.
int enqueue_xy(Plan* P, const unsigned long long* gq, const unsigned long long* gq2, const float* gf,
               cudaStream_t s, bool events);
ZParams zparams(const Plan* P, int mode);
int finish_power(Plan* P, cudaStream_t s, fkp_power_out* out, bool have_scalars, double I22, double N0);
int bisp_plan_init(Plan* P);
void bisp_plan_free(Plan* P);
// Frees the plan's bispectrum graph (its buffers changed, or graphs were
// turned off); the next repeat of a call captures a new one.
void bisp_drop_graph(Plan* P);
// Records a stage event on s; inside a stream capture as an external event
// node, so that a replayed graph still times its stages.
cudaError_t record_stage(cudaEvent_t ev, cudaStream_t s);

// launch wrappers (k_power.cu)
int yz_tiles(int N);
int tiles_x(int N);
bool moments_match(const MomentTable& mt);
size_t field_elems(int N);
cudaError_t launch_scalars_finalize(const double* part, int nbg, int nbr, long long ng, long long nr, int amode,
                                    double* ds, cudaStream_t s);
int assign_tiles_per_axis(int N);
cudaError_t launch_bin_count(const CatDev& c, int is_ran, const GeomDev& g, double* part, int* bh, int* err,
                             int nblk, cudaStream_t s);
cudaError_t launch_tile_prefix(int* bh, int nrows, int ntiles, int* cnt, cudaStream_t s);
cudaError_t launch_scan_tiles(const int* cnt, int ntiles, int* off, int* items, cudaStream_t s);
cudaError_t launch_bin_scatter(const CatDev& c, int is_ran, const GeomDev& g, const double obs[3], const double* ds,
                               const int* off, const int* bpref, float4* xyzv, float* vw2, double* labpart, int nblk,
                               cudaStream_t s, int raw = 0);
cudaError_t launch_combine_randoms(unsigned long long* grid, const unsigned long long* rgrid,
                                   unsigned long long* gridw, const unsigned long long* rgridw, const double* ds,
                                   long long n, int nsm, cudaStream_t s);
// xe: NULL, or the exponents (a, b, c) of a moment field: each object's value
// is then multiplied by x^_x^a x^_y^b x^_z^c of its own line of sight.
cudaError_t launch_tile_accum(const GeomDev& g, const int* off, const int* items, long long nobj, const float4* xyzv,
                              const float* vw2, unsigned long long* grid, unsigned long long* gridw, cudaStream_t s,
                              const unsigned char* xe = nullptr);
cudaError_t launch_lab_finalize(const double* labpart, int nblk, double* out, cudaStream_t s);
cudaError_t launch_wait_selftest(unsigned polls, int* flag, cudaStream_t s);
// xm: x-pass blocks = SMs x resident blocks x xm; nt: threads per y- or
// z-pass block (256 or 512).  The defaults are the 512^3 choices.  mb: the
// mocks of one fused launch (blockIdx.z) and their buffer strides.
// per_object: gq holds mt.nfields gridded moment fields one after the other
// (N^3 each); the x-pass transforms them instead of forming the moments at
// the nodes.
cudaError_t launch_xpass(const unsigned long long* gq, const float* gf, const GeomDev& g, const MomentTable& mt,
                         const FftPlan& fp, const float2* tw, float2* S1, int nsm, cudaStream_t s, int xm = 2,
                         MockBatch mb = MockBatch(), bool per_object = false);
cudaError_t launch_ypass(const float2* S1, const unsigned long long* gq, const float* gf, const GeomDev& g,
                         const MomentTable& mt, const FftPlan& fp,
                         const float2* tw, float2* S2, int* err, cudaStream_t s, int nt = 256,
                         MockBatch mb = MockBatch());
// The z-pass is persistent: zpass_blocks(N, nt, nsm) blocks, each writing
// one column of the partial bins (part[key][block]); reduce over that count.
cudaError_t launch_zpass(const float2* S2, const GeomDev& g, const MomentTable& mt, const FftPlan& fp,
                         const float2* tw, const ZParams& zp, double* part, int* partc, int* err, cudaStream_t s,
                         int nsm, int nt = 512, MockBatch mb = MockBatch());
int zpass_blocks(int N, int nt, int nsm);
cudaError_t launch_reduce_bins(const double* part, const int* partc, int nblk, int nbins, double* out,
                               long long* outc, cudaStream_t s, int nmock = 1, long long pstride = 0,
                               long long pcstride = 0);

// tensor-core triangle contraction (k_contract_tc.cu)
void tc_slicing(long long N3, int ntiles, int nsm, int* nslices, int* chunks);
int tc_tile_cols();
int tc_rows();
cudaError_t launch_contract_tc(const float* I, long long N3, int nf, int S, const short2* pairs, int npairs,
                               float* part, int* err, int nslices, int chunks, int nsplit, cudaStream_t s);
cudaError_t launch_tc_reduce(const float* part, int nslices, int ntiles, const int* om, const int* on, int nout,
                             double* out, cudaStream_t s);

}  // namespace fkp
