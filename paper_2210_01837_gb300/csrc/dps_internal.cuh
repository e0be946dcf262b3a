// Internal declarations of the GB300 doubly-periodic FCM mobility library.
// Everything here is private to the library; the public C ABI is include/dpstokes.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/dpstokes.h"

namespace dps {

// ---------------------------------------------------------------------------------------------
// complex helpers (interleaved re/im, 8- or 16-byte aligned)
// ---------------------------------------------------------------------------------------------
template <typename T> struct cplx;
template <> struct __align__(8) cplx<float> { float x, y; };
template <> struct __align__(16) cplx<double> { double x, y; };

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T a, T b) { cplx<T> r; r.x = a; r.y = b; return r; }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __host__ __device__ __forceinline__ cplx<T> scl(cplx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
template <typename T> __host__ __device__ __forceinline__ cplx<T> conjg(cplx<T> a) { return mk<T>(a.x, -a.y); }
// multiply by i
template <typename T> __host__ __device__ __forceinline__ cplx<T> mul_i(cplx<T> a) { return mk<T>(-a.y, a.x); }

// ---------------------------------------------------------------------------------------------
// tiling constants
// ---------------------------------------------------------------------------------------------
constexpr int kTileX = 32;          // spread tile / particle bin, nodes in x
constexpr int kTileY = 8;           // nodes in y
constexpr int kSpreadThreads = kTileX * kTileY;
constexpr int kMaxFftRadices = 24;
constexpr int kMaxM = 12;           // largest ES support in cells
constexpr int kBvpThreads = 128;    // threads (wavenumbers) per block in the per-k solver
constexpr int kMaxChunks = 16;      // column chunks of the wavenumber-space pipeline
constexpr int kMaxTimed = 8 + 5 * kMaxChunks;  // timed launches per apply

// FFT factorisation (radices applied in order, Stockham autosort)
struct FftPlan {
  int n;
  int nstages;
  int radix[kMaxFftRadices];
  unsigned long long magic[kMaxFftRadices];  // floor(2^40 / Ns) + 1 for the span Ns of each stage
  int toff[kMaxFftRadices];  // stage s >= 1: offset of its twiddles W_{Ns R}^{k r}, [k < Ns][r < R], in the
                             // stage-twiddle table (tab.tsy, read by the column passes); total length in toff[0]
};

// Per-kernel (monopole / dipole) ES parameters on the device
struct EsKernel {
  double alpha;     // support half width
  double beta;      // shape
  double inv_norm;  // 1 / integral of exp(beta (sqrt(1-(t/alpha)^2) - 1)) over [-alpha, alpha]
  double cut;       // derivative kernel: phi'(t) = 0 for |t| > cut (kernel-derivative torque route)
  int px;           // x/y node slots per particle (m + 1)
  // float copies for the float evaluations (a division or conversion in double at every
  // evaluation would occupy the FP64 pipe): 1/alpha, beta, 1/Z, beta/alpha
  float inv_alpha_f, beta_f, inv_norm_f, beta_over_alpha_f;
};

// Everything a kernel needs to know about the problem (passed by value)
struct Geometry {
  double Lx, Ly, zmin, zmax, H, h, inv_h;
  double sH, inv_eta;  // 2 / H and 1 / eta (host divisions, so the solves do not repeat them)
  double eta;
  int mode;          // dps_wall_mode
  int nx, ny, nz;
  int nkx;           // nx/2 + 1
  int pitch;         // complex elements per stored row (>= nkx); real rows hold 2*pitch values
  int nfields;       // fields spread and transformed: 6 (spectral-curl torques) or 3
  int with_torque;   // applies take torques and return angular velocities
  int spectral_curl; // torque fields are spread; the half-curl is taken in Fourier-Chebyshev space
  int torque_deriv;  // the half-curl of the dipole envelope is spread with the forces; Omega by
                     // interpolation with the envelope gradient
  int nbx, nby;      // bins (spread tiles) in x and y
  int rbx, rby;      // bin radius searched around a tile
  EsKernel kM, kD;
  int pxc;           // x/y slots in a particle record (max over kernels)
  int lzc;           // z slots in a particle record
  int rec_words;     // 32-bit words per particle record
  int nkernels;      // 1 (M) or 2 (M and D): record heads
  int nslabs;        // value slabs per record: one per kernel, plus the dipole derivative slab
  // wall conditions beyond no-slip stationary walls (Appendix A): slip lengths and uniform
  // tangential wall velocities; slip = 1 when any of them is non-zero
  double slip0, slipH;
  double uw0[2], uwH[2];
  int slip;
  int stage_cap;     // particle records the spreading kernel stages in shared memory at a time
  int rec_threads;   // threads per block of the record kernel when it stages records in shared
                     // memory (0: direct writes)
};

// Device tables owned by the plan
struct Tables {
  double* zc;      // [nz] node heights, c = 0 at zmax
  void* wz;        // [nz] T Clenshaw-Curtis weights (times h^2 is applied in interpolation)
  void* zeta;      // [nz] T  z_c - zmin
  double* band;    // [5][nz] doubles: l_n, d_n, u_n, P_n, Q_n of the spectral-integration operator
  void* twx;       // [nx] cplx<T>  exp(-2 pi i t / nx)
  void* twy;       // [ny] cplx<T>  exp(-2 pi i t / ny)
  void* tsy;       // cplx<T> stage twiddles of the register-staged y passes (Plan::fyr, FftPlan::toff)
};

// per-wavenumber stage: transform tables (T, padded for vector loads) and buffers
struct KTabs {
  void* ct;        // [N][npad]  forward DCT-I, transposed: ct[c][n] = C[n][c]
  void* dct;       // [N][npad]  (2/H) D C transposed
  void* ict;       // [N][cpad]  inverse DCT-I transposed: ict[n][c] = IC[c][n]
  void* icdt;      // [N][cpad]  (2/H) IC D transposed (derivative at the nodes from coefficients)
  void* sdt;       // [N][cpad]  spectral differentiation at the nodes, transposed: sdt[j][c] = SD[c][j]
  void* bandT;     // [3][N]     l, d, u of the B B map in T
  void* cmat;      // [N][N]     forward DCT-I C[n][j] (correction coefficients in the tiled backward)
  void* kbuf;      // [3][N][K]  Chebyshev coefficients per wavenumber (forces, then DP velocity)
  void* kaux;      // [12][K]    wall-correction amplitudes per wavenumber
  double* fac;     // [N][4][KP] factorisation of the banded systems per (kx, |ky|) (FP64), or null
  int64_t KP;      // nkx (ny/2 + 1)
  unsigned char* bimg_f;  // tensor-core transforms: B operands of every K step (forward, backward)
  unsigned char* bimg_b;
  int npad, cpad;
  int fwd_smem, bwd_smem;
};

struct Plan {
  int device;
  int precision;        // dps_precision
  int64_t max_n;
  Geometry g;
  FftPlan fx, fy;
  FftPlan fxr, fyr;     // x / y transforms of the register-staged passes (balanced factorisation)
  Tables tab;
  KTabs kt;
  // device buffers
  void* grid;           // [nfields][nz][ny][pitch] cplx<T> (real rows: 2*pitch T)
  uint32_t* records;    // [max_n][rec_words]
  int* bin_of;          // [max_n]
  int* bin_count;       // [nbins]
  int* bin_start;       // [nbins + 1]
  int* bin_cursor;      // [nbins]
  int* sorted;          // [max_n]
  int* zrange;          // [2] occupied Chebyshev plane range (c_lo, c_hi)
  int* status;          // [1] device status bits
  void* ws;             // per-slot workspace of the per-k solver
  int bvp_blocks;       // persistent grid size of the per-k solver
  int fft_grid[4];      // resident grids of the persistent FFT passes: rows fwd/inv, columns fwd/inv
  int col_lcw;          // log2 of the column block of the y-FFT pass (default rule or autotuned)
  int fft_reg[2];       // FFT variant of the row and the column pass: 0 smem-staged, 1 register-staged,
                        // 2 (columns) register-staged with cp.async prefetch, 3 (columns) the same with
                        // TMA box loads
  alignas(64) unsigned char col_tmap[128];  // CUtensorMap of the grid for the TMA column pass
  alignas(64) unsigned char interp_tmap[128];  // CUtensorMap of the grid for the staged interpolation
  int interp_tma;       // interp_tmap holds a valid map
  int col_tma_rows;     // rows per TMA box of that pass
  int bvp_blocks_max;   // persistent solve blocks the workspace was allocated for
  int interp_tile;      // interpolation variant: 0 warp per particle, 1 tile gather, 2 staged grid (where they apply)
  int cheb_tc;          // forward Chebyshev transform on the tensor cores (tcgen05, mixed precision)
  int cheb_tc_bwd;      // backward Chebyshev transform on the tensor cores (spectral-curl torques)
  int cheb_tc_bwd_parts;  // launches of the backward transform (output planes split beyond 96 nodes)
  int cheb_tc_grid;     // persistent blocks of that kernel
  int inject;           // failure injection of the next apply (dpstokes_debug_inject)
  void* ipart;          // partial sums of the tile-gather interpolation [slot][field][max_n] T
  int64_t ws_bytes;
  // host-input staging (dpstokes_apply_host)
  double* stage_in;     // [max_n][9]
  double* stage_out;    // [max_n][6]
  int64_t device_bytes;
  // wavenumber-space pipeline: column chunks on three streams (fork/join by events)
  int nchunks;
  int chunk_x0[kMaxChunks + 1];
  cudaStream_t side[2];
  cudaEvent_t ev_fork, ev_f[kMaxChunks], ev_s[kMaxChunks], ev_b[kMaxChunks];
  // per-stage timing (dpstokes_enable_timing): a start/end event pair per launch, summed per stage
  int timing;
  int timed_apply;
  int nev;
  int ev_stage[kMaxTimed];
  cudaEvent_t ev0[kMaxTimed], ev1[kMaxTimed];
};

// ---------------------------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async): the issuing thread continues at once and
// cp_wait_all() later waits for its own copies (a __syncthreads() then publishes them), so a block
// can keep many copies in flight without holding registers for them.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async8(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async4(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// wait until at most the newest committed group of this thread is still in flight
__device__ __forceinline__ void cp_wait_but_newest() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// one naturally aligned element of 4, 8 or 16 bytes
template <typename E>
__device__ __forceinline__ void async_elem(E* s, const E* g) {
  static_assert(sizeof(E) == 4 || sizeof(E) == 8 || sizeof(E) == 16, "cp.async sizes");
  if (sizeof(E) == 16) cp_async16(s, g);
  else if (sizeof(E) == 8) cp_async8(s, g);
  else cp_async4(s, g);
}

// The largest dynamic shared memory a kernel may be launched with is an attribute of the kernel,
// shared by every plan in the process.  Raising it once to what the device allows (minus the
// kernel's static shared memory) lets plans of different sizes coexist; the bytes each launch asks
// for still decide occupancy.
template <typename K>
inline bool allow_smem(K kernel) {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return false;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes) == cudaSuccess;
}

// float -> double with integer operations only (a conversion instruction would occupy the FP64
// pipe, which this GPU has little of); exact for normal numbers, infinities and NaNs; float
// subnormals become zero.
__device__ __forceinline__ double widen_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  if (e == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
  const unsigned m = b & 0x7fffffu;
  const unsigned de = (e == 0xffu) ? 0x7ffu : e + 896u;
  return __hiloint2double((int)((b & 0x80000000u) | (de << 20) | (m >> 3)), (int)(m << 29));
}

// double -> float with integer operations only, rounding toward zero (|result| <= |d|); exact
// exponent handling for normal floats, results below the float normal range become zero, above it
// infinity (NaN inputs are not expected: callers check finiteness first).
__device__ __forceinline__ float narrow_bits(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned s = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;
  if (e <= 0) return __uint_as_float(s);
  if (e >= 255) return __uint_as_float(s | 0x7f800000u);
  return __uint_as_float(s | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// status bits written by kernels
enum : int { kStatNonfinite = 1, kStatDomain = 2, kStatInternal = 4, kStatTimeout = 8 };

// host side of the particle stage: the ES normalisation (Eq. 54), the truncation point of the
// derivative kernel, and the particle-side geometry (kernels, record layout, bins) shared by plans
// and the allocation-free spread; g must hold the box, grid and wall mode.  tsize: 32-bit words
// per stored value (1 float, 2 double).
double es_norm(double alpha, double beta);
double es_deriv_cut(double alpha, double beta);
dps_status particle_geometry(Geometry& g, const dps_kernel_params* kp, int tsize);

// launchers (stream-ordered, no host sync)
template <typename T> void launch_records(const Plan& p, int64_t n, const double* pos, const double* F,
                                          const double* Tq, cudaStream_t s);
void launch_bins(const Plan& p, int64_t n, cudaStream_t s);
template <typename T> void launch_spread(const Plan& p, cudaStream_t s);
template <typename T> int spread_prepare(Plan& p);  // 1 ready, 0 CUDA error, -1 records too large
template <typename T> void launch_interp(const Plan& p, int64_t n, double* U, double* W, cudaStream_t s);
// the tile-gather interpolation: fields it sums for this geometry (0: it does not apply) and the
// values of its partial-sum buffer for max_n particles
int interp_tile_fields(const Geometry& g);
// the staged-grid interpolation (variant 2): fields it sums for this geometry and transform
// precision (tsize 32-bit words per value), 0 where it does not apply
int interp_stage_fields(const Geometry& g, int tsize);
// encodes the staged interpolation's tensor map of the grid (float plans); false when the driver's
// encoder cannot be obtained or refuses the map
bool encode_interp_tmap(Plan& p);
size_t interp_tile_values(const Geometry& g, int64_t max_n);
template <typename T> void launch_fft_rows(const Plan& p, int dir, cudaStream_t s);
template <typename T> void launch_fft_cols(const Plan& p, int dir, int kxs, int kxe, cudaStream_t s);
template <typename T> int fft_col_width(const Plan& p);
// part 0 Chebyshev forward, 1 FP64 solve, 2 backward; columns [kx0, kx0 + w) of every ky
template <typename T> void launch_bvp(const Plan& p, int part, int kx0, int w, cudaStream_t s);
template <typename T> int bvp_occupancy_blocks(const Plan& p);
template <typename T> int bvp_prepare(Plan& p);
// the factorisation table of the FP64 solve (allocated and filled at plan creation); DPS_ERR_OOM
// leaves the plan on the factorise-as-you-go solve
dps_status bvp_factor_table(Plan& p);
// the tensor-core forward Chebyshev transform: readiness (sets cheb_tc where it applies; 0 on a CUDA
// error), its launcher, and its accumulator width (nz rounded up to 16)
int cheb_tc_prepare(Plan& p);
void launch_cheb_fwd_tc(const Plan& p, int kx0, int w, cudaStream_t s);
void launch_cheb_bwd_tc(const Plan& p, int kx0, int w, cudaStream_t s);
int cheb_tc_np(const Geometry& g);
size_t cheb_tc_image_bytes(const Geometry& g, bool backward);
template <typename T> size_t bvp_slot_bytes(const Plan& p);
template <typename T> int fft_smem_ok(Plan& p);
// column block 2^lcw and variant of the y-FFT pass (reg: 0 shared-memory-staged, 1 register-staged,
// 2 register-staged with cp.async prefetch, 3 register-staged with TMA prefetch); 0 if it does not fit
template <typename T> int fft_set_col_width(Plan& p, int lcw, int reg);
// x-FFT pass variant: register-staged (reg = 1) or shared-memory-staged; 0 if it does not fit
template <typename T> int fft_set_row_variant(Plan& p, int reg);

// host-side validation of an apply's arguments, and the stream-ordered product itself
dps_status check_apply_args(const Plan* p, int64_t n, const double* pos, const double* F, const double* Tq,
                            const double* U, const double* W, bool need_out = true);
dps_status run(Plan* p, int64_t n, const double* pos, const double* F, const double* Tq, double* U, double* W,
               cudaStream_t s, int last_stage);

}  // namespace dps
