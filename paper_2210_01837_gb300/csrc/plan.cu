// Host side of the library: plan construction (validation, tables, device buffers), the apply
// pipeline (steps 1-8 of Sec. III.D enqueued on one stream) and the C ABI of include/dpstokes.h.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "dps_internal.cuh"

namespace dps {
namespace {

bool smooth_7(int n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5, 7})
    while (n % p == 0) n /= p;
  return n == 1;
}

// stage constants of a plan whose radices are set: per-stage magic numbers and twiddle-row offsets
void fft_plan_finish(FftPlan& fp) {
  unsigned long long ns = 1;
  int off = 0;
  for (int s = 0; s < fp.nstages; ++s) {
    fp.magic[s] = (1ull << 40) / ns + 1;
    if (s > 0) {
      fp.toff[s] = off;
      off += ((int)ns * fp.radix[s] + 1) & ~1;  // even offsets: float rows of even R stay 16-byte aligned
    }
    ns *= (unsigned long long)fp.radix[s];
  }
  fp.toff[0] = off;
}

// Greedy factorisation, largest radices first (the shared-memory-staged passes).
bool fft_plan(int n, FftPlan& fp) {
  fp.n = n;
  fp.nstages = 0;
  int m = n;
  while (m % 16 == 0 && fp.nstages < kMaxFftRadices) { fp.radix[fp.nstages++] = 16; m /= 16; }
  while (m % 12 == 0 && fp.nstages < kMaxFftRadices) { fp.radix[fp.nstages++] = 12; m /= 12; }
  while (m % 8 == 0 && fp.nstages < kMaxFftRadices) { fp.radix[fp.nstages++] = 8; m /= 8; }
  while (m % 4 == 0 && fp.nstages < kMaxFftRadices) { fp.radix[fp.nstages++] = 4; m /= 4; }
  while (m % 2 == 0 && fp.nstages < kMaxFftRadices) { fp.radix[fp.nstages++] = 2; m /= 2; }
  for (int p : {3, 5, 7})
    while (m % p == 0 && fp.nstages < kMaxFftRadices) { fp.radix[fp.nstages++] = p; m /= p; }
  fft_plan_finish(fp);
  return m == 1 && n < (1 << 20);
}

// Balanced factorisation (the register-staged passes, one butterfly per thread and stage, so their
// thread count is n / (smallest radix)): the fewest stages, then the largest smallest radix, radices
// in descending order.  768 = 12 8 8 instead of 16 16 3, 384 = 12 8 4 instead of 16 12 2.
namespace {
const int kRadices[] = {16, 12, 8, 7, 5, 4, 3, 2};
void balanced_search(int m, int from, int* cur, int depth, int* best, int& best_depth, int& best_min) {
  if (m == 1) {
    int mn = 1 << 30;
    for (int i = 0; i < depth; ++i) mn = std::min(mn, cur[i]);
    if (depth < best_depth || (depth == best_depth && mn > best_min)) {
      best_depth = depth;
      best_min = mn;
      for (int i = 0; i < depth; ++i) best[i] = cur[i];
    }
    return;
  }
  if (depth >= best_depth || depth >= kMaxFftRadices) return;
  for (int k = from; k < 8; ++k)
    if (m % kRadices[k] == 0) {
      cur[depth] = kRadices[k];
      balanced_search(m / kRadices[k], k, cur, depth + 1, best, best_depth, best_min);
    }
}
}  // namespace

bool fft_plan_balanced(int n, FftPlan& fp) {
  if (!fft_plan(n, fp)) return false;  // the greedy plan: validity and a fallback
  int cur[kMaxFftRadices], best[kMaxFftRadices];
  int best_depth = kMaxFftRadices + 1, best_min = 0;
  balanced_search(n, 0, cur, 0, best, best_depth, best_min);
  if (best_depth > kMaxFftRadices || best_depth > fp.nstages) return true;
  fp.nstages = best_depth;
  for (int i = 0; i < best_depth; ++i) fp.radix[i] = best[i];
  fft_plan_finish(fp);
  return true;
}

template <typename T>
cudaError_t upload(void** dst, const std::vector<double>& v, int64_t& bytes) {
  std::vector<T> h(v.begin(), v.end());
  cudaError_t e = cudaMalloc(dst, std::max<size_t>(1, h.size() * sizeof(T)));
  if (e != cudaSuccess) return e;
  bytes += (int64_t)(h.size() * sizeof(T));
  return cudaMemcpy(*dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

template <typename T>
cudaError_t upload_twiddles(void** dst, int n, int64_t& bytes) {
  std::vector<T> h(2 * (size_t)n);
  for (int t = 0; t < n; ++t) {
    // exp(-2 pi i t / n), argument reduced to t/n in [0, 1)
    const double a = -2.0 * M_PI * (double)t / (double)n;
    h[2 * t] = (T)cos(a);
    h[2 * t + 1] = (T)sin(a);
  }
  cudaError_t e = cudaMalloc(dst, h.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  bytes += (int64_t)(h.size() * sizeof(T));
  return cudaMemcpy(*dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Stage twiddles: for each stage s >= 1 (span Ns, radix R) the values W_{Ns R}^{k r} =
// exp(-2 pi i k r / (Ns R)), k < Ns, r < R, row k contiguous, so a butterfly reads its R twiddles
// from one row instead of R scattered entries of the length-n table.
template <typename T>
cudaError_t upload_stage_twiddles(void** dst, const FftPlan& fp, int64_t& bytes) {
  std::vector<T> h(2 * (size_t)std::max(fp.toff[0], 1), (T)0);
  int ns = 1;
  for (int s = 0; s < fp.nstages; ++s) {
    const int R = fp.radix[s];
    if (s > 0) {
      for (int k = 0; k < ns; ++k)
        for (int r = 0; r < R; ++r) {
          const long long m = ((long long)k * r) % ((long long)ns * R);  // argument reduced to [0, 1)
          const double a = -2.0 * M_PI * (double)m / ((double)ns * R);
          const size_t i = (size_t)fp.toff[s] + (size_t)k * R + r;
          h[2 * i] = (T)cos(a);
          h[2 * i + 1] = (T)sin(a);
        }
    }
    ns *= R;
  }
  cudaError_t e = cudaMalloc(dst, h.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  bytes += (int64_t)(h.size() * sizeof(T));
  return cudaMemcpy(*dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

__global__ void apply_init_kernel(int* zrange, int nz, int* bin_count, int nbins) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    zrange[0] = nz;
    zrange[1] = -1;
  }
  for (int b = i; b < nbins; b += gridDim.x * blockDim.x) bin_count[b] = 0;
}

void free_plan(Plan* p) {
  if (!p) return;
  for (int i = 0; i < kMaxTimed; ++i) {
    if (p->ev0[i]) cudaEventDestroy(p->ev0[i]);
    if (p->ev1[i]) cudaEventDestroy(p->ev1[i]);
  }
  for (int j = 0; j < kMaxChunks; ++j) {
    if (p->ev_f[j]) cudaEventDestroy(p->ev_f[j]);
    if (p->ev_s[j]) cudaEventDestroy(p->ev_s[j]);
    if (p->ev_b[j]) cudaEventDestroy(p->ev_b[j]);
  }
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  for (int i = 0; i < 2; ++i)
    if (p->side[i]) cudaStreamDestroy(p->side[i]);
  void* ptrs[] = {p->tab.zc, p->tab.wz, p->tab.zeta, p->tab.band, p->tab.twx, p->tab.twy, p->tab.tsy,
                  p->kt.ct, p->kt.dct,
                  p->kt.ict, p->kt.icdt, p->kt.sdt, p->kt.bandT, p->kt.cmat, p->kt.kbuf, p->kt.kaux, p->grid, p->records, p->bin_of, p->bin_count, p->bin_start,
                  p->bin_cursor, p->sorted, p->zrange, p->status, p->ws, p->stage_in, p->stage_out, p->ipart,
                  p->kt.fac, p->kt.bimg_f, p->kt.bimg_b};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete p;
}

template <typename T>
dps_status build_tables(Plan* p) {
  const Geometry& g = p->g;
  const int N = g.nz;
  const int n1 = N - 1;
  int64_t& bytes = p->device_bytes;
  // Chebyshev extrema nodes, c = 0 at zmax
  std::vector<double> zc(N), zeta(N);
  for (int c = 0; c < N; ++c) {
    zc[c] = g.zmin + 0.5 * g.H * (1.0 + cos(M_PI * c / n1));
    zeta[c] = zc[c] - g.zmin;
  }
  // forward DCT-I: a_n = (2/n1) sum'' g_c cos(pi n c / n1), a_0 and a_n1 halved; inverse IC[c][n]
  std::vector<double> C((size_t)N * N), IC((size_t)N * N);
  for (int n = 0; n < N; ++n)
    for (int c = 0; c < N; ++c) {
      const double cs = cos(M_PI * (double)((int64_t)n * c % (2 * n1)) / n1);
      double v = 2.0 / n1 * cs;
      if (c == 0 || c == n1) v *= 0.5;
      if (n == 0 || n == n1) v *= 0.5;
      C[(size_t)n * N + c] = v;
      IC[(size_t)c * N + n] = cs;
    }
  // Chebyshev derivative matrix Dm[m][n] (coefficient m of d/ds T_n) by the recurrence
  // b_m = b_{m+2} + 2 (m+1) a_{m+1}, b_0 halved
  std::vector<double> Dm((size_t)N * N, 0.0);
  for (int n = 0; n < N; ++n) {
    std::vector<double> b(N + 2, 0.0);
    for (int m = N - 2; m >= 0; --m) b[m] = b[m + 2] + ((m + 1 == n) ? 2.0 * (m + 1) : 0.0);
    b[0] *= 0.5;
    for (int m = 0; m < N; ++m) Dm[(size_t)m * N + n] = b[m];
  }
  const double sH = 2.0 / g.H;
  std::vector<double> DC((size_t)N * N, 0.0), ICD((size_t)N * N, 0.0), SD((size_t)N * N, 0.0);
  for (int m = 0; m < N; ++m)
    for (int c = 0; c < N; ++c) {
      double s1 = 0.0, s2 = 0.0;
      for (int q = 0; q < N; ++q) {
        s1 += Dm[(size_t)m * N + q] * C[(size_t)q * N + c];   // (D C)[m][c]
        s2 += IC[(size_t)c * N + q] * Dm[(size_t)q * N + m];  // (IC D)[c][m]
      }
      DC[(size_t)m * N + c] = sH * s1;
      ICD[(size_t)c * N + m] = sH * s2;
    }
  for (int c = 0; c < N; ++c)
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
      for (int q = 0; q < N; ++q) s += ICD[(size_t)c * N + q] * C[(size_t)q * N + j];
      SD[(size_t)c * N + j] = s;
    }
  const int npad = (N + 24 + 3) / 4 * 4, cpad = (N + 8 + 3) / 4 * 4;
  p->kt.npad = npad;
  p->kt.cpad = cpad;
  std::vector<double> ct((size_t)N * npad, 0.0), dct((size_t)N * npad, 0.0);
  std::vector<double> ict((size_t)N * cpad, 0.0), icdt((size_t)N * cpad, 0.0), sdt((size_t)N * cpad, 0.0);
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      ct[(size_t)a * npad + b] = C[(size_t)b * N + a];     // [c][n]
      dct[(size_t)a * npad + b] = DC[(size_t)b * N + a];
      ict[(size_t)a * cpad + b] = IC[(size_t)b * N + a];   // [n][c]
      icdt[(size_t)a * cpad + b] = ICD[(size_t)b * N + a];
      sdt[(size_t)a * cpad + b] = SD[(size_t)b * N + a];   // [j][c]
    }
  // Clenshaw-Curtis weights: integral of the interpolant, w = C^T I, I_n = 2/(1-n^2) (n even)
  std::vector<double> wz(N, 0.0);
  for (int c = 0; c < N; ++c) {
    double s = 0.0;
    for (int n = 0; n < N; n += 2) s += C[(size_t)n * N + c] * 2.0 / (1.0 - (double)n * n);
    wz[c] = 0.5 * g.H * s;
  }
  // banded spectral-integration operator: (B B c)_m = l_m c_{m-2} + d_m c_m + u_m c_{m+2}
  std::vector<double> band(5 * (size_t)N, 0.0);
  double* l = band.data();
  double* d = l + N;
  double* u = d + N;
  double* P = u + N;
  double* Q = P + N;
  for (int m = 1; m < N; ++m) {
    if (m == 1) { l[m] = 0.0; d[m] = -1.0 / 8.0; u[m] = 1.0 / 8.0; }
    else if (m == 2) { l[m] = 0.25; d[m] = -1.0 / 6.0; u[m] = 1.0 / 24.0; }
    else { l[m] = 1.0 / (4.0 * m * (m - 1)); d[m] = -1.0 / (2.0 * ((double)m * m - 1.0)); u[m] = 1.0 / (4.0 * m * (m + 1)); }
    if (m + 2 >= N) u[m] = 0.0;
  }
  // column sums: Q_j = sum_m BB[m][j], P_j = sum_m m^2 BB[m][j]
  for (int j = 0; j < N; ++j) {
    double q = d[j], pp = (double)j * j * d[j];
    if (j + 2 < N) { q += l[j + 2]; pp += (double)(j + 2) * (j + 2) * l[j + 2]; }
    if (j - 2 >= 0) { q += u[j - 2]; pp += (double)(j - 2) * (j - 2) * u[j - 2]; }
    Q[j] = q;
    P[j] = pp;
  }
  cudaError_t e = cudaSuccess;
  if ((e = upload<double>((void**)&p->tab.zc, zc, bytes)) != cudaSuccess) return DPS_ERR_OOM;
  if ((e = upload<double>((void**)&p->tab.band, band, bytes)) != cudaSuccess) return DPS_ERR_OOM;
  if ((e = upload<T>(&p->tab.wz, wz, bytes)) != cudaSuccess) return DPS_ERR_OOM;
  if ((e = upload<T>(&p->kt.ct, ct, bytes)) != cudaSuccess) return DPS_ERR_OOM;
  if ((e = upload<T>(&p->kt.dct, dct, bytes)) != cudaSuccess) return DPS_ERR_OOM;
  if ((e = upload<T>(&p->kt.ict, ict, bytes)) != cudaSuccess) return DPS_ERR_OOM;
  if ((e = upload<T>(&p->kt.icdt, icdt, bytes)) != cudaSuccess) return DPS_ERR_OOM;
  if ((e = upload<T>(&p->kt.sdt, sdt, bytes)) != cudaSuccess) return DPS_ERR_OOM;
  if ((e = upload<T>(&p->kt.cmat, C, bytes)) != cudaSuccess) return DPS_ERR_OOM;
  {
    std::vector<double> bt(3 * (size_t)N);
    for (size_t i = 0; i < 3 * (size_t)N; ++i) bt[i] = band[i];
    if ((e = upload<T>(&p->kt.bandT, bt, bytes)) != cudaSuccess) return DPS_ERR_OOM;
  }
  if ((e = upload<T>(&p->tab.zeta, zeta, bytes)) != cudaSuccess) return DPS_ERR_OOM;
  if ((e = upload_twiddles<T>(&p->tab.twx, g.nx, bytes)) != cudaSuccess) return DPS_ERR_OOM;
  if ((e = upload_twiddles<T>(&p->tab.twy, g.ny, bytes)) != cudaSuccess) return DPS_ERR_OOM;
  if ((e = upload_stage_twiddles<T>(&p->tab.tsy, p->fyr, bytes)) != cudaSuccess) return DPS_ERR_OOM;
  return DPS_OK;
}

// column chunks of the wavenumber-space pipeline: multiples of 32 columns; false if too narrow
bool set_chunks(Plan& p, int J) {
  const int nkx = p.g.nkx;
  if (J < 1 || J > kMaxChunks || (J > 1 && nkx < 64 * J)) return false;
  p.nchunks = J;
  for (int j = 0; j < J; ++j) p.chunk_x0[j] = (int)((int64_t)j * nkx / J) / 32 * 32;
  p.chunk_x0[J] = nkx;
  return true;
}

template <typename T>
dps_status allocate(Plan* p) {
  Geometry& g = p->g;
  int64_t& bytes = p->device_bytes;
  auto alloc = [&](void** q, size_t sz) -> bool {
    if (cudaMalloc(q, std::max<size_t>(sz, 16)) != cudaSuccess) return false;
    bytes += (int64_t)sz;
    return true;
  };
  const size_t nmax = (size_t)std::max<int64_t>(p->max_n, 1);
  const int nbins = g.nbx * g.nby;
  if (!alloc(&p->grid, (size_t)g.nfields * g.nz * g.ny * g.pitch * sizeof(cplx<T>))) return DPS_ERR_OOM;
  if (!alloc((void**)&p->records, nmax * g.rec_words * sizeof(uint32_t))) return DPS_ERR_OOM;
  if (!alloc((void**)&p->bin_of, nmax * sizeof(int))) return DPS_ERR_OOM;
  if (!alloc((void**)&p->sorted, nmax * sizeof(int))) return DPS_ERR_OOM;
  if (!alloc((void**)&p->bin_count, (size_t)nbins * sizeof(int))) return DPS_ERR_OOM;
  if (!alloc((void**)&p->bin_start, (size_t)(nbins + 1) * sizeof(int))) return DPS_ERR_OOM;
  if (!alloc((void**)&p->bin_cursor, (size_t)nbins * sizeof(int))) return DPS_ERR_OOM;
  if (!alloc((void**)&p->zrange, 2 * sizeof(int))) return DPS_ERR_OOM;
  if (!alloc((void**)&p->status, sizeof(int))) return DPS_ERR_OOM;
  if (cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) return DPS_ERR_CUDA;
  p->bvp_blocks = bvp_occupancy_blocks<T>(*p);
  const int64_t K = (int64_t)g.nkx * g.ny;
  const int64_t need_blocks = (K + kBvpThreads - 1) / kBvpThreads;
  if (p->bvp_blocks > need_blocks) p->bvp_blocks = (int)std::max<int64_t>(1, need_blocks);
  p->bvp_blocks_max = p->bvp_blocks;
  p->ws_bytes = (int64_t)p->bvp_blocks * kBvpThreads * (int64_t)bvp_slot_bytes<T>(*p);
  if (!alloc(&p->ws, (size_t)p->ws_bytes)) return DPS_ERR_OOM;
  if (!alloc(&p->kt.kbuf, 3 * (size_t)g.nz * (size_t)K * sizeof(cplx<T>))) return DPS_ERR_OOM;
  if (!alloc(&p->kt.kaux, 12 * (size_t)K * sizeof(cplx<T>))) return DPS_ERR_OOM;
  if (!bvp_prepare<T>(*p)) return DPS_ERR_INVALID_ARG;
  if (!cheb_tc_prepare(*p)) return DPS_ERR_CUDA;
  if (p->cheb_tc && !alloc((void**)&p->kt.bimg_f, cheb_tc_image_bytes(g, false))) return DPS_ERR_OOM;
  if (p->cheb_tc_bwd && !alloc((void**)&p->kt.bimg_b, cheb_tc_image_bytes(g, true))) return DPS_ERR_OOM;
  if (const char* e = getenv("DPS_CHEB_TC")) {  // bit 0 forward, bit 1 backward
    const int v = atoi(e);
    p->cheb_tc = p->cheb_tc && (v & 1);
    p->cheb_tc_bwd = p->cheb_tc_bwd && (v & 2);
  }
  // factorisation table of the FP64 solve (per (kx, |ky|), filled on the legacy stream): without
  // the memory for it the solve factorises as it goes; DPS_SOLVE_TABLE=0 chooses that by hand
  {
    const char* e = getenv("DPS_SOLVE_TABLE");
    if (!(e && atoi(e) == 0)) {
      const dps_status ft = bvp_factor_table(*p);
      if (ft == DPS_ERR_CUDA) return ft;
    }
  }
  // the tile-gather interpolation's partial sums (where it applies; a variant the autotuner tries)
  if (const size_t iv = interp_tile_values(g, p->max_n)) {
    if (!alloc(&p->ipart, iv * sizeof(T))) return DPS_ERR_OOM;
  }
  // default: the staged gather where it applies, else a warp per particle; the autotuner tries the
  // others
  p->interp_tile = interp_stage_fields(g, (int)(sizeof(T) / 4)) > 0 ? 2 : 0;
  if (const char* e = getenv("DPS_INTERP_TILE")) {
    p->interp_tile = 0;
    const int v = atoi(e);
    if (v == 1 && p->ipart) p->interp_tile = 1;
    if (v == 2 && interp_stage_fields(g, (int)(sizeof(T) / 4)) > 0) p->interp_tile = 2;
  }
  if (!alloc((void**)&p->stage_in, nmax * 9 * sizeof(double))) return DPS_ERR_OOM;
  if (!alloc((void**)&p->stage_out, nmax * 6 * sizeof(double))) return DPS_ERR_OOM;
  if (!fft_smem_ok<T>(*p)) return DPS_ERR_INVALID_ARG;
  const int sp = spread_prepare<T>(*p);
  if (sp < 0) return DPS_ERR_INVALID_ARG;
  if (sp == 0) return DPS_ERR_CUDA;
  // the staged interpolation's TMA view of the grid (without it every bin copies with cp.async)
  p->interp_tma = interp_stage_fields(g, (int)(sizeof(T) / 4)) > 0 && encode_interp_tmap(*p) ? 1 : 0;
  // column chunks of the wavenumber-space pipeline (multiples of 32 columns, ~192 wide)
  // one chunk by default: measured on GB300, co-running the FP64 solve with the float transforms
  // slowed both (they compete for issue slots); DPS_CHUNKS in the environment or the autotuner may
  // choose more
  int J = 1;
  if (const char* e = getenv("DPS_CHUNKS")) J = std::max(1, std::min(atoi(e), kMaxChunks));
  if (!set_chunks(*p, J)) set_chunks(*p, 1);
  for (int i = 0; i < 2; ++i)
    if (cudaStreamCreateWithFlags(&p->side[i], cudaStreamNonBlocking) != cudaSuccess) return DPS_ERR_CUDA;
  if (cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess) return DPS_ERR_CUDA;
  for (int j = 0; j < kMaxChunks; ++j) {  // events for every chunk count the autotuner may pick
    if (cudaEventCreateWithFlags(&p->ev_f[j], cudaEventDisableTiming) != cudaSuccess) return DPS_ERR_CUDA;
    if (cudaEventCreateWithFlags(&p->ev_s[j], cudaEventDisableTiming) != cudaSuccess) return DPS_ERR_CUDA;
    if (cudaEventCreateWithFlags(&p->ev_b[j], cudaEventDisableTiming) != cudaSuccess) return DPS_ERR_CUDA;
  }
  return DPS_OK;
}

template <typename T>
void enqueue(Plan& p, int64_t n, const double* pos, const double* F, const double* Tq, double* U, double* W,
             cudaStream_t s, int last_stage) {
  const int nbins = p.g.nbx * p.g.nby;
  const bool tm = p.timing != 0 && last_stage >= 6;
  p.nev = 0;
  // bracket one launch with a timed event pair on the stream it runs on
  auto timed = [&](int stage, cudaStream_t st, auto&& launch) {
    const int i = p.nev;
    if (tm && i < kMaxTimed) cudaEventRecord(p.ev0[i], st);
    launch();
    if (tm && i < kMaxTimed) {
      cudaEventRecord(p.ev1[i], st);
      p.ev_stage[i] = stage;
      p.nev = i + 1;
    }
  };
  timed(0, s, [&] {
    apply_init_kernel<<<std::min(1024, (nbins + 255) / 256 + 1), 256, 0, s>>>(p.zrange, p.g.nz, p.bin_count, nbins);
  });
  timed(1, s, [&] { launch_records<T>(p, n, pos, F, Tq, s); });
  if (last_stage <= 1) return;
  timed(2, s, [&] { launch_bins(p, n, s); });
  timed(3, s, [&] { launch_spread<T>(p, s); });
  if (last_stage <= 2) return;
  timed(4, s, [&] { launch_fft_rows<T>(p, -1, s); });
  if (last_stage <= 3) {
    launch_fft_cols<T>(p, -1, 0, p.g.nkx, s);
    return;
  }
  // wavenumber space, column chunks: y-FFT + Chebyshev forward on s, FP64 solve on side[0],
  // backward + inverse y-FFT on side[1]; the FP64-bound solve of one chunk overlaps the float and
  // memory-bound work of its neighbours
  cudaStream_t ss = p.side[0], sb = p.side[1];
  cudaEventRecord(p.ev_fork, s);
  cudaStreamWaitEvent(ss, p.ev_fork, 0);
  cudaStreamWaitEvent(sb, p.ev_fork, 0);
  const bool inverse = last_stage >= 5;
  for (int j = 0; j < p.nchunks; ++j) {
    const int x0 = p.chunk_x0[j], x1 = p.chunk_x0[j + 1];
    timed(5, s, [&] { launch_fft_cols<T>(p, -1, x0, x1, s); });
    timed(6, s, [&] { launch_bvp<T>(p, 0, x0, x1 - x0, s); });
    cudaEventRecord(p.ev_f[j], s);
    cudaStreamWaitEvent(ss, p.ev_f[j], 0);
    timed(7, ss, [&] { launch_bvp<T>(p, 1, x0, x1 - x0, ss); });
    cudaEventRecord(p.ev_s[j], ss);
    cudaStreamWaitEvent(sb, p.ev_s[j], 0);
    timed(8, sb, [&] { launch_bvp<T>(p, 2, x0, x1 - x0, sb); });
    if (inverse) timed(9, sb, [&] { launch_fft_cols<T>(p, +1, x0, x1, sb); });
    cudaEventRecord(p.ev_b[j], sb);
  }
  cudaStreamWaitEvent(s, p.ev_b[p.nchunks - 1], 0);
  cudaStreamWaitEvent(s, p.ev_s[p.nchunks - 1], 0);
  if (!inverse) return;
  timed(10, s, [&] { launch_fft_rows<T>(p, +1, s); });
  if (last_stage <= 5) return;
  timed(11, s, [&] { launch_interp<T>(p, n, U, W, s); });
  if (tm) p.timed_apply = 1;
  p.inject = 0;  // an injected failure applies to one apply
}

}  // namespace

dps_status check_apply_args(const Plan* p, int64_t n, const double* pos, const double* F, const double* Tq,
                            const double* U, const double* W, bool need_out) {
  if (!p || n < 0 || n > p->max_n) return DPS_ERR_INVALID_ARG;
  if (n > 0 && (!pos || !F || (need_out && !U))) return DPS_ERR_INVALID_ARG;
  if (p->g.with_torque) {
    if (n > 0 && (!Tq || (need_out && !W))) return DPS_ERR_INVALID_ARG;
  } else if (Tq || W) {
    return DPS_ERR_INVALID_ARG;
  }
  return DPS_OK;
}

dps_status run(Plan* p, int64_t n, const double* pos, const double* F, const double* Tq, double* U, double* W,
               cudaStream_t s, int last_stage) {
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) cudaSetDevice(p->device);
  if (p->precision == DPS_MIXED)
    enqueue<float>(*p, n, pos, F, Tq, U, W, s, last_stage);
  else
    enqueue<double>(*p, n, pos, F, Tq, U, W, s, last_stage);
  const cudaError_t e = cudaGetLastError();
  if (dev != p->device && dev >= 0) cudaSetDevice(dev);
  return e == cudaSuccess ? DPS_OK : DPS_ERR_CUDA;
}

}  // namespace dps

using dps::Plan;

extern "C" {

const char* dpstokes_error_string(dps_status st) {
  switch (st) {
    case DPS_OK: return "ok";
    case DPS_ERR_INVALID_ARG: return "invalid argument";
    case DPS_ERR_OUT_OF_DOMAIN: return "particle height outside the domain or envelope through an open boundary";
    case DPS_ERR_OOM: return "device allocation failed";
    case DPS_ERR_CUDA: return "CUDA runtime error";
    case DPS_ERR_TIMEOUT: return "bounded device wait expired";
    case DPS_ERR_NONFINITE: return "non-finite input";
    case DPS_ERR_BUSY: return "server queue at its limit: request not accepted";
  }
  return "unknown status";
}

dps_status dpstokes_plan_create(dps_plan_t* out, double Lx, double Ly, double zmin, double zmax, int32_t wall_mode,
                                const dps_grid* grid, const dps_kernel_params* kp) {
  return dpstokes_plan_create_ex(out, Lx, Ly, zmin, zmax, wall_mode, grid, kp, nullptr);
}

dps_status dpstokes_plan_create_ex(dps_plan_t* out, double Lx, double Ly, double zmin, double zmax, int32_t wall_mode,
                                   const dps_grid* grid, const dps_kernel_params* kp, const dps_wall_params* wp) {
  if (!out) return DPS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!grid || !kp) return DPS_ERR_INVALID_ARG;
  if (!(Lx > 0) || !(Ly > 0) || !(zmax > zmin) || !isfinite(Lx) || !isfinite(Ly) || !isfinite(zmin) || !isfinite(zmax))
    return DPS_ERR_INVALID_ARG;
  if (wall_mode < DPS_FREE || wall_mode > DPS_SLIT) return DPS_ERR_INVALID_ARG;
  const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
  if (nx < 8 || ny < 8 || nz < 5 || nz > 257 || !dps::smooth_7(nx) || !dps::smooth_7(ny)) return DPS_ERR_INVALID_ARG;
  const double hx = Lx / nx, hy = Ly / ny;
  if (fabs(hx - hy) > 1e-12 * hx) return DPS_ERR_INVALID_ARG;
  if (kp->precision != DPS_FP64 && kp->precision != DPS_MIXED) return DPS_ERR_INVALID_ARG;
  if (kp->max_n < 0 || kp->max_n > (int64_t)1 << 30) return DPS_ERR_INVALID_ARG;
  if (!(kp->eta > 0) || !isfinite(kp->eta)) return DPS_ERR_INVALID_ARG;
  dps::Geometry g;
  memset(&g, 0, sizeof(g));
  g.Lx = Lx; g.Ly = Ly; g.zmin = zmin; g.zmax = zmax; g.H = zmax - zmin; g.sH = 2.0 / g.H;
  g.h = hx; g.inv_h = 1.0 / hx; g.eta = kp->eta; g.inv_eta = 1.0 / kp->eta; g.mode = wall_mode;
  g.nx = nx; g.ny = ny; g.nz = nz; g.nkx = nx / 2 + 1;
  g.pitch = (g.nkx + 31) / 32 * 32;
  // kernels, torque route, particle records and bins
  const int tsize = (kp->precision == DPS_FP64) ? 2 : 1;  // 32-bit words per stored value
  if (dps::particle_geometry(g, kp, tsize) != DPS_OK) return DPS_ERR_INVALID_ARG;
  if (wp) {
    const double v[6] = {wp->slip_bottom, wp->slip_top, wp->uw_bottom[0], wp->uw_bottom[1], wp->uw_top[0],
                         wp->uw_top[1]};
    for (double x : v)
      if (!isfinite(x)) return DPS_ERR_INVALID_ARG;
    if (wp->slip_bottom < 0.0 || wp->slip_top < 0.0) return DPS_ERR_INVALID_ARG;
    const bool bottom = wall_mode == DPS_BOTTOM_WALL || wall_mode == DPS_SLIT, top = wall_mode == DPS_SLIT;
    if (!bottom && (wp->slip_bottom != 0.0 || wp->uw_bottom[0] != 0.0 || wp->uw_bottom[1] != 0.0))
      return DPS_ERR_INVALID_ARG;
    if (!top && (wp->slip_top != 0.0 || wp->uw_top[0] != 0.0 || wp->uw_top[1] != 0.0)) return DPS_ERR_INVALID_ARG;
    g.slip0 = wp->slip_bottom;
    g.slipH = wp->slip_top;
    g.uw0[0] = wp->uw_bottom[0];
    g.uw0[1] = wp->uw_bottom[1];
    g.uwH[0] = wp->uw_top[0];
    g.uwH[1] = wp->uw_top[1];
    for (double x : v) g.slip = g.slip || x != 0.0;
  }

  Plan* p = new (std::nothrow) Plan();
  if (!p) return DPS_ERR_OOM;
  memset(p, 0, sizeof(Plan));
  cudaGetDevice(&p->device);
  p->precision = kp->precision;
  p->max_n = kp->max_n;
  p->g = g;
  if (!dps::fft_plan(nx, p->fx) || !dps::fft_plan(ny, p->fy) || !dps::fft_plan_balanced(nx, p->fxr) ||
      !dps::fft_plan_balanced(ny, p->fyr)) {
    dps::free_plan(p);
    return DPS_ERR_INVALID_ARG;
  }
  dps_status st = (p->precision == DPS_MIXED) ? dps::build_tables<float>(p) : dps::build_tables<double>(p);
  if (st == DPS_OK) st = (p->precision == DPS_MIXED) ? dps::allocate<float>(p) : dps::allocate<double>(p);
  if (st != DPS_OK) { dps::free_plan(p); cudaGetLastError(); return st; }
  // the uploads and clears ran on the legacy stream; waiting for it leaves work on non-blocking
  // streams (other plans' applies, the serving slots) running
  if (cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess) { dps::free_plan(p); cudaGetLastError(); return DPS_ERR_CUDA; }
  *out = reinterpret_cast<dps_plan_t>(p);
  return DPS_OK;
}

dps_status dpstokes_apply(dps_plan_t plan, int64_t n, const double* positions, const double* forces,
                          const double* torques, double* out_vel, double* out_angvel, void* stream) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  const dps_status st = dps::check_apply_args(p, n, positions, forces, torques, out_vel, out_angvel);
  if (st != DPS_OK) return st;
  return dps::run(p, n, positions, forces, torques, out_vel, out_angvel, (cudaStream_t)stream, 99);
}

dps_status dpstokes_apply_host(dps_plan_t plan, int64_t n, const double* positions, const double* forces,
                               const double* torques, double* out_vel, double* out_angvel, void* stream) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  dps_status st = dps::check_apply_args(p, n, positions, forces, torques, out_vel, out_angvel);
  if (st != DPS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  double* dpos = p->stage_in;
  double* dF = dpos + 3 * (size_t)p->max_n;
  double* dT = p->g.with_torque ? dF + 3 * (size_t)p->max_n : nullptr;
  double* dU = p->stage_out;
  double* dW = p->g.with_torque ? dU + 3 * (size_t)p->max_n : nullptr;
  const size_t b = 3 * (size_t)n * sizeof(double);
  if (n > 0) {
    if (cudaMemcpyAsync(dpos, positions, b, cudaMemcpyHostToDevice, s) != cudaSuccess) return DPS_ERR_CUDA;
    if (cudaMemcpyAsync(dF, forces, b, cudaMemcpyHostToDevice, s) != cudaSuccess) return DPS_ERR_CUDA;
    if (dT && cudaMemcpyAsync(dT, torques, b, cudaMemcpyHostToDevice, s) != cudaSuccess) return DPS_ERR_CUDA;
  }
  st = dps::run(p, n, dpos, dF, dT, dU, dW, s, 99);
  if (st != DPS_OK) return st;
  if (n > 0) {
    if (cudaMemcpyAsync(out_vel, dU, b, cudaMemcpyDeviceToHost, s) != cudaSuccess) return DPS_ERR_CUDA;
    if (dW && cudaMemcpyAsync(out_angvel, dW, b, cudaMemcpyDeviceToHost, s) != cudaSuccess) return DPS_ERR_CUDA;
  }
  return dpstokes_status(plan, stream);
}

dps_status dpstokes_status(dps_plan_t plan, void* stream) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p) return DPS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DPS_ERR_CUDA;
  int v = 0;
  if (cudaMemcpy(&v, p->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DPS_ERR_CUDA;
  if (v != 0 && cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) return DPS_ERR_CUDA;
  if (v & dps::kStatNonfinite) return DPS_ERR_NONFINITE;
  if (v & dps::kStatDomain) return DPS_ERR_OUT_OF_DOMAIN;
  if (v & dps::kStatInternal) return DPS_ERR_CUDA;
  if (v & dps::kStatTimeout) return DPS_ERR_TIMEOUT;
  return DPS_OK;
}

void dpstokes_destroy(dps_plan_t plan) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p) return;
  cudaDeviceSynchronize();
  dps::free_plan(p);
}

dps_status dpstokes_plan_info(dps_plan_t plan, dps_plan_info* out) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !out) return DPS_ERR_INVALID_ARG;
  out->device_bytes = p->device_bytes;
  out->nkx = p->g.nkx;
  out->pitch = p->g.pitch;
  out->nfields = p->g.nfields;
  out->record_words = p->g.rec_words;
  out->h = p->g.h;
  out->alpha_M = p->g.kM.alpha;
  out->alpha_D = p->g.with_torque ? p->g.kD.alpha : 0.0;
  // init, records, 3 binning, spread, x pass, 5 per column chunk, x pass, interpolation (+ its
  // finishing kernel for the tile gather)
  // (+ the B-operand image kernel before each tensor-core transform)
  out->launches_per_apply = 9 + 5 * p->nchunks + ((p->interp_tile == 1 && p->ipart) ? 1 : 0) +
                            p->nchunks * ((p->cheb_tc ? 1 : 0) + (p->cheb_tc_bwd ? 2 * p->cheb_tc_bwd_parts - 1 : 0));
  out->nchunks = p->nchunks;
  out->fft_col_width = 1 << p->col_lcw;
  out->fft_register_rows = p->fft_reg[0];
  out->fft_register_cols = p->fft_reg[1];
  out->solve_blocks = p->bvp_blocks;
  out->interp_variant = p->interp_tile;
  out->cheb_tensor_cores = (p->cheb_tc ? 1 : 0) | (p->cheb_tc_bwd ? 2 : 0);
  return DPS_OK;
}

dps_status dpstokes_debug_inject(dps_plan_t plan, int32_t code) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || code < 0 || code > 3 || (code == 1 && !p->cheb_tc) || (code == 2 && p->interp_tile != 2) ||
      (code == 3 && p->fft_reg[1] != 3))
    return DPS_ERR_INVALID_ARG;
  p->inject = code;
  return DPS_OK;
}

dps_status dpstokes_plan_set_interp(dps_plan_t plan, int32_t variant) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || variant < 0 || variant > 2) return DPS_ERR_INVALID_ARG;
  if (variant == 1 && !p->ipart) return DPS_ERR_INVALID_ARG;
  if (variant == 2 && dps::interp_stage_fields(p->g, p->precision == DPS_FP64 ? 2 : 1) == 0) return DPS_ERR_INVALID_ARG;
  p->interp_tile = variant;
  return DPS_OK;
}

dps_status dpstokes_plan_autotune(dps_plan_t plan, int64_t n, const double* positions, const double* forces,
                                  const double* torques, double* out_vel, double* out_angvel, void* stream,
                                  double* best_ms) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  dps_status st = dps::check_apply_args(p, n, positions, forces, torques, out_vel, out_angvel);
  if (st != DPS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return DPS_ERR_CUDA;
  // mean time of two applies after one untimed apply
  auto measure = [&](double* ms) -> dps_status {
    dps_status r = dps::run(p, n, positions, forces, torques, out_vel, out_angvel, s, 99);
    if (r != DPS_OK) return r;
    cudaEventRecord(e0, s);
    for (int i = 0; i < 2 && r == DPS_OK; ++i) r = dps::run(p, n, positions, forces, torques, out_vel, out_angvel, s, 99);
    cudaEventRecord(e1, s);
    if (r != DPS_OK) return r;
    if (cudaEventSynchronize(e1) != cudaSuccess) return DPS_ERR_CUDA;
    float f = 0.f;
    if (cudaEventElapsedTime(&f, e0, e1) != cudaSuccess) return DPS_ERR_CUDA;
    *ms = 0.5 * f;
    return DPS_OK;
  };
  const bool mixed = p->precision == DPS_MIXED;
  auto set_width = [&](int l, int reg) {
    return mixed ? dps::fft_set_col_width<float>(*p, l, reg) : dps::fft_set_col_width<double>(*p, l, reg);
  };
  double best = 0.0, t = 0.0;
  st = measure(&best);
  // keep a candidate only when it is clearly (2 %) faster than the incumbent
  auto better = [&](double cand) { return cand < 0.98 * best; };
  // 1. column block and variant (register- or shared-memory-staged) of the y-FFT pass
  int best_l = p->col_lcw, best_r = p->fft_reg[1];
  for (int r = 3; r >= 0 && st == DPS_OK; --r)
    for (int l = 0; l <= 3 && st == DPS_OK; ++l) {
      if ((l == best_l && r == best_r) || !set_width(l, r)) continue;
      st = measure(&t);
      if (st == DPS_OK && better(t)) { best = t; best_l = l; best_r = r; }
    }
  set_width(best_l, best_r);
  // 2. persistent grid of the FP64 solve (blocks per SM, within the allocated workspace)
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  int best_b = p->bvp_blocks;
  for (int per = 1; per <= 4 && st == DPS_OK; ++per) {
    const int b = std::min(per * sms, p->bvp_blocks_max);
    if (b == best_b) continue;
    p->bvp_blocks = b;
    st = measure(&t);
    if (st == DPS_OK && better(t)) { best = t; best_b = b; }
  }
  p->bvp_blocks = best_b;
  // 3. column chunks of the wavenumber-space pipeline (the FP64 solve of one chunk overlaps the
  //    float transforms of its neighbours)
  int best_j = p->nchunks;
  for (int j : {1, 2, 4}) {
    if (st != DPS_OK) break;
    if (j == best_j || !dps::set_chunks(*p, j)) continue;
    st = measure(&t);
    if (st == DPS_OK && better(t)) { best = t; best_j = j; }
  }
  dps::set_chunks(*p, best_j);
  // 4. interpolation variant (tile gather or warp per particle), where both apply
  {
    const int inc = p->interp_tile;
    int best_v = inc;
    for (int v = 0; v < 3 && st == DPS_OK; ++v) {
      if (v == inc || (v == 1 && !p->ipart) ||
          (v == 2 && dps::interp_stage_fields(p->g, p->precision == DPS_FP64 ? 2 : 1) == 0))
        continue;
      p->interp_tile = v;
      st = measure(&t);
      if (st == DPS_OK && better(t)) { best = t; best_v = v; }
    }
    p->interp_tile = best_v;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DPS_OK) return st;
  // leave the outputs holding the product with the chosen shapes
  st = dps::run(p, n, positions, forces, torques, out_vel, out_angvel, s, 99);
  if (st != DPS_OK) return st;
  if (best_ms) *best_ms = best;
  return dpstokes_status(plan, stream);
}

dps_status dpstokes_plan_set_fft(dps_plan_t plan, int32_t row_register, int32_t col_register, int32_t col_width) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || (row_register != 0 && row_register != 1) || col_register < 0 || col_register > 3)
    return DPS_ERR_INVALID_ARG;
  int l = -1;
  for (int k = 0; k <= 3; ++k)
    if (col_width == (1 << k)) l = k;
  if (l < 0) return DPS_ERR_INVALID_ARG;
  const bool mixed = p->precision == DPS_MIXED;
  const int old_reg[2] = {p->fft_reg[0], p->fft_reg[1]}, old_l = p->col_lcw;
  auto set_rows = [&](int r) { return mixed ? dps::fft_set_row_variant<float>(*p, r) : dps::fft_set_row_variant<double>(*p, r); };
  auto set_cols = [&](int k, int r) {
    return mixed ? dps::fft_set_col_width<float>(*p, k, r) : dps::fft_set_col_width<double>(*p, k, r);
  };
  if (set_rows(row_register) && set_cols(l, col_register)) return DPS_OK;
  set_rows(old_reg[0]);
  set_cols(old_l, old_reg[1]);
  return DPS_ERR_INVALID_ARG;
}

dps_status dpstokes_plan_set_pipeline(dps_plan_t plan, int32_t solve_blocks, int32_t nchunks) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || solve_blocks < 1 || solve_blocks > p->bvp_blocks_max) return DPS_ERR_INVALID_ARG;
  if (nchunks != 1 && nchunks != 2 && nchunks != 4 && nchunks != 8) return DPS_ERR_INVALID_ARG;
  const int old = p->nchunks;
  if (!dps::set_chunks(*p, nchunks)) {
    dps::set_chunks(*p, old);
    return DPS_ERR_INVALID_ARG;
  }
  p->bvp_blocks = solve_blocks;
  return DPS_OK;
}

dps_status dpstokes_enable_timing(dps_plan_t plan, int32_t enable) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p) return DPS_ERR_INVALID_ARG;
  if (enable && !p->ev0[0]) {
    for (int i = 0; i < dps::kMaxTimed; ++i) {
      if (cudaEventCreate(&p->ev0[i]) != cudaSuccess) return DPS_ERR_CUDA;
      if (cudaEventCreate(&p->ev1[i]) != cudaSuccess) return DPS_ERR_CUDA;
    }
  }
  p->timing = enable ? 1 : 0;
  p->timed_apply = 0;
  return DPS_OK;
}

dps_status dpstokes_stage_times(dps_plan_t plan, double* ms_out, int32_t capacity, int32_t* count) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !ms_out || capacity < 0 || !p->timing || !p->timed_apply) return DPS_ERR_INVALID_ARG;
  double acc[DPS_NUM_STAGES] = {0.0};
  for (int i = 0; i < p->nev; ++i) {
    if (cudaEventSynchronize(p->ev1[i]) != cudaSuccess) return DPS_ERR_CUDA;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p->ev0[i], p->ev1[i]) != cudaSuccess) return DPS_ERR_CUDA;
    acc[p->ev_stage[i]] += ms;
  }
  const int m = std::min<int>(capacity, DPS_NUM_STAGES);
  for (int i = 0; i < m; ++i) ms_out[i] = acc[i];
  if (count) *count = m;
  return DPS_OK;
}

dps_status dpstokes_debug_run(dps_plan_t plan, int64_t n, const double* positions, const double* forces,
                              const double* torques, double* out_vel, double* out_angvel, void* stream,
                              int32_t last_stage) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (last_stage < 1 || last_stage > 6) return DPS_ERR_INVALID_ARG;
  const dps_status st = dps::check_apply_args(p, n, positions, forces, torques, out_vel, out_angvel, last_stage >= 6);
  if (st != DPS_OK) return st;
  return dps::run(p, n, positions, forces, torques, out_vel, out_angvel, (cudaStream_t)stream, last_stage);
}

dps_status dpstokes_debug_copy(dps_plan_t plan, int32_t which, void* dst, int64_t dst_bytes, void* stream) {
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (!p || !dst || dst_bytes < 0) return DPS_ERR_INVALID_ARG;
  const size_t tsz = p->precision == DPS_MIXED ? sizeof(float) : sizeof(double);
  const void* src = nullptr;
  size_t sz = 0;
  if (which == 0) { src = p->grid; sz = (size_t)p->g.nfields * p->g.nz * p->g.ny * p->g.pitch * 2 * tsz; }
  else if (which == 1) { src = p->records; sz = (size_t)std::max<int64_t>(p->max_n, 1) * p->g.rec_words * 4; }
  else if (which == 2) { src = p->zrange; sz = 2 * sizeof(int); }
  else return DPS_ERR_INVALID_ARG;
  sz = std::min(sz, (size_t)dst_bytes);
  if (cudaMemcpyAsync(dst, src, sz, cudaMemcpyDeviceToDevice, (cudaStream_t)stream) != cudaSuccess) return DPS_ERR_CUDA;
  return DPS_OK;
}

}  // extern "C"
