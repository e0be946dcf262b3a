// Forward Chebyshev transform (step 2 of Sec. III.D, z part, with the half-curl source of the
// torque route) on the 5th-generation tensor cores.
//
// Per wavenumber k the transform is a contraction over the occupied planes c:
//   out_o[n] = sum_c C[n][c] a_o(c) + DC[n][c] b_o(c),   o = 0, 1, 2,
// with a_o = f_o + (1/2)(i k x tau)_o, b_x = -tau_y/2, b_y = tau_x/2, b_z = 0 (C the DCT-I,
// DC = (2/H) D C).  Real and imaginary parts contract independently, so a block takes 64
// wavenumbers as the M = 128 rows of a GEMM (row 2j + p: wavenumber j, part p), the planes as K
// and the Chebyshev index n as N (padded to Np, a multiple of 16):
//   D_o[128 x Np] += A_o[128 x 8] B[8 x Np] per chunk of 8 planes (tcgen05.mma .kind::tf32, the
// accumulators of the three outputs side by side in tensor memory).  Float accuracy from tf32
// operands by the three-product split: x = x_hi + x_lo with x_hi = tf32(x), x_lo = tf32(x - x_hi),
// and A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped A_lo B_lo is 2^-22 relative).
//
// A block is persistent over 64-wavenumber tiles.  The CUDA cores build each plane chunk's
// operands (grid values with the curl terms; table rows of C and DC), split them, and store them
// in the K-major core-matrix layout into one of two shared-memory stages; one thread issues the
// chunk's MMAs and commits them to that stage's mbarrier, and the other threads go on building the
// next chunk in the other stage.  After the last chunk the accumulators are read with tcgen05.ld
// and written to kbuf[o][n][k] (a warp's 32 lanes hold 16 wavenumbers' real and imaginary parts,
// contiguous in kbuf).  Every mbarrier wait is bounded (about a second); on expiry the block
// records DPS_ERR_TIMEOUT in the status word, waits once more (bounded) for its issued MMAs,
// frees its tensor memory and leaves.
#include <math.h>

#include <algorithm>

#include "dps_internal.cuh"
#include "umma_desc.h"

namespace dps {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcRows = 128;   // MMA M: 64 wavenumbers x (re, im)
constexpr int kTcK = 8;        // planes per K step (8 tf32 = 32 bytes per operand row)
constexpr int kTcWave = 64;    // wavenumbers per tile
constexpr long long kWaitCycles = 1ll << 31;  // bounded waits: about one second at 2 GHz

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

// wait until the phase of the given parity has completed; false after kWaitCycles
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

// 8 consecutive 32-bit columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void split4(float4 v, float4& hi, float4& lo) {
  hi = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
  lo = make_float4(tf32_rna(v.x - hi.x), tf32_rna(v.y - hi.y), tf32_rna(v.z - hi.z), tf32_rna(v.w - hi.w));
}

// shared-memory stage: A tiles [NQ][hi, lo][128 rows x 8], B tiles [NT][hi, lo][Np rows x 8]
struct TcStage {
  static constexpr uint32_t kATile = kTcRows * kTcK * 4;  // 4096 bytes
  __host__ __device__ static uint32_t bytes(int nq, int nt, int np) {
    return (uint32_t)(2 * nq * kATile + 2 * nt * np * kTcK * 4);
  }
};

// thread i of a chunk (columns [kx0, kx0 + w), every ky) -> wavenumber index kyi * nkx + kxi
__device__ __forceinline__ int64_t tc_kidx(const Geometry& g, int64_t i, int kx0, int w) {
  const unsigned ii = (unsigned)i;
  const int kyi = (int)(ii / (unsigned)w);
  return (int64_t)kyi * g.nkx + kx0 + (int)(ii - (unsigned)kyi * (unsigned)w);
}

template <bool CURL>
__global__ void __launch_bounds__(kTcThreads, 2) cheb_fwd_tc_kernel(Geometry g, const float* __restrict__ ct,
                                                                    const float* __restrict__ dct, int npad,
                                                                    const cplx<float>* __restrict__ grid,
                                                                    cplx<float>* __restrict__ kbuf,
                                                                    const int* __restrict__ zrange, int kx0, int w,
                                                                    int np, int tcols, int* __restrict__ status) {
  constexpr int NQ = CURL ? 5 : 3;  // A operands per chunk: a0, b0, a1, b1, a2 (forces only: a0, a1, a2)
  constexpr int NT = CURL ? 2 : 1;  // B operands: C (and DC)
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_col[kTcWave], s_kid[kTcWave];
  __shared__ float s_hkx[kTcWave], s_hky[kTcWave];
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = g.nz;
  const int clo = zrange[0], chi = zrange[1];
  const int64_t K = (int64_t)g.nkx * g.ny;
  const int64_t total = (int64_t)w * g.ny;
  const int64_t ntiles = (total + kTcWave - 1) / kTcWave;
  const uint32_t stage_bytes = TcStage::bytes(NQ, NT, np);
  const uint32_t btile = (uint32_t)np * kTcK * 4;
  unsigned char* stage0 = smraw;
  const size_t plane = (size_t)g.ny * g.pitch;
  const size_t fstride = (size_t)g.nz * plane;
  const uint32_t idesc = umma::idesc_tf32(kTcRows, (uint32_t)np);
  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&s_tmem, (uint32_t)tcols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  unsigned uses[2] = {0, 0};  // completed-or-issued commits per stage (uniform across the block)
  const int nchunks = chi >= clo ? (chi - clo + kTcK) / kTcK : 0;
  bool ok = true;
  for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    if (tid < kTcWave) {
      const int64_t it = tile * kTcWave + tid;
      int col = -1, kid = 0;
      float hx = 0.f, hy = 0.f;
      if (it < total) {
        const int64_t kidx = tc_kidx(g, it, kx0, w);
        const unsigned ku = (unsigned)kidx;
        const int kyi = (int)(ku / (unsigned)g.nkx), kxi = (int)(ku - (unsigned)kyi * (unsigned)g.nkx);
        const int nyv = (kyi < (g.ny + 1) / 2) ? kyi : kyi - g.ny;
        col = kyi * g.pitch + kxi;
        kid = (int)kidx;
        hx = (float)(M_PI * (double)kxi / g.Lx);
        hy = (float)(M_PI * (double)nyv / g.Ly);
      }
      s_col[tid] = col;
      s_kid[tid] = kid;
      s_hkx[tid] = hx;
      s_hky[tid] = hy;
    }
    __syncthreads();
    // thread (j, grp, half): wavenumber j, planes 4 grp .. 4 grp + 3 of each chunk; half 0 builds
    // a0, b0, a1 (forces only: a0, a1), half 1 builds b1, a2 (forces only: a2).  The grid values of
    // chunk q + 1 are loaded into registers before chunk q's operands are stored, so their latency
    // overlaps the barrier and the MMA issue.
    const int j = tid & 63, grp = (tid >> 6) & 1, half = tid >> 7;
    const int jcol = s_col[j];
    const float hkx = s_hkx[j], hky = s_hky[j];
    constexpr int NR = CURL ? 4 : 2;  // grid fields read per plane by this thread
    cplx<float> raw[4][NR];
    auto load = [&](int q) {
      const int c0 = clo + q * kTcK;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int c = c0 + 4 * grp + cc;
        const bool in = jcol >= 0 && c <= chi;
        const cplx<float>* p = grid + (size_t)c * plane + (in ? jcol : 0);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          // half 0 reads fx, fy, ty, tz (forces only: fx, fy); half 1 reads fz, tx, ty (fz)
          const int f = CURL ? (half == 0 ? (r < 2 ? r : r + 2) : (r < 3 ? r + 2 : 4)) : (half == 0 ? r : 2);
          raw[cc][r] = in && (half == 0 || r < (CURL ? 3 : 1)) ? p[(size_t)f * fstride] : mk<float>(0.f, 0.f);
        }
      }
    };
    if (nchunks > 0) load(0);
    for (int q = 0; q < nchunks; ++q) {
      const int sb = q & 1;
      unsigned char* st = stage0 + sb * stage_bytes;
      // the MMAs that last read this stage must have completed
      if (uses[sb] > 0 && !mbar_wait(&s_bar[sb], (uses[sb] - 1) & 1)) {
        if (tid == 0) s_fail = 1;
      }
      __syncthreads();
      if (s_fail) { ok = false; break; }
      const int c0 = clo + q * kTcK;
      {
        float re[3][4], im[3][4];
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          if (CURL) {
            if (half == 0) {
              const cplx<float> fx = raw[cc][0], fy = raw[cc][1], ty = raw[cc][2], tz = raw[cc][3];
              // a0 = fx + i ky/2 tz, b0 = -ty/2, a1 = fy - i kx/2 tz
              re[0][cc] = fx.x - hky * tz.y;  im[0][cc] = fx.y + hky * tz.x;
              re[1][cc] = -0.5f * ty.x;       im[1][cc] = -0.5f * ty.y;
              re[2][cc] = fy.x + hkx * tz.y;  im[2][cc] = fy.y - hkx * tz.x;
            } else {
              const cplx<float> fz = raw[cc][0], tx = raw[cc][1], ty = raw[cc][2];
              // b1 = tx/2, a2 = fz + i (kx/2 ty - ky/2 tx)
              const float sx = hkx * ty.x - hky * tx.x, sy = hkx * ty.y - hky * tx.y;
              re[0][cc] = 0.5f * tx.x;        im[0][cc] = 0.5f * tx.y;
              re[1][cc] = fz.x - sy;          im[1][cc] = fz.y + sx;
              re[2][cc] = 0.f;                im[2][cc] = 0.f;
            }
          } else {
            re[0][cc] = raw[cc][0].x;  im[0][cc] = raw[cc][0].y;
            re[1][cc] = raw[cc][1].x;  im[1][cc] = raw[cc][1].y;
            re[2][cc] = 0.f;           im[2][cc] = 0.f;
          }
        }
        if (q + 1 < nchunks) load(q + 1);
        // operand index of each built quantity
        const int nb = CURL ? (half == 0 ? 3 : 2) : (half == 0 ? 2 : 1);
        const int first = half == 0 ? 0 : (CURL ? 3 : 2);
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          if (u >= nb) break;
          const int qi = first + u;
          unsigned char* ahi = st + (size_t)(2 * qi) * TcStage::kATile;
          unsigned char* alo = ahi + TcStage::kATile;
#pragma unroll
          for (int pp = 0; pp < 2; ++pp) {
            const uint32_t off = umma::kmajor_offset((uint32_t)(2 * j + pp), (uint32_t)(4 * grp));
            const float(&x)[4] = pp ? im[u] : re[u];
            float4 hi, lo;
            split4(make_float4(x[0], x[1], x[2], x[3]), hi, lo);
            *reinterpret_cast<float4*>(ahi + off) = hi;
            *reinterpret_cast<float4*>(alo + off) = lo;
          }
        }
      }
      // ---- B: thread (n, group, table): C[n][c] (and DC[n][c]) for four planes
      for (int item = tid; item < np * 2 * NT; item += kTcThreads) {
        const int n = item % np, grp = (item / np) & 1, tab = item / (2 * np);
        const float* src = tab == 0 ? ct : dct;
        float x[4];
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const int c = c0 + 4 * grp + cc;
          x[cc] = (n < N && c <= chi) ? src[(size_t)c * npad + n] : 0.f;
        }
        float4 hi, lo;
        split4(make_float4(x[0], x[1], x[2], x[3]), hi, lo);
        unsigned char* bt = st + (size_t)2 * NQ * TcStage::kATile + (size_t)(2 * tab) * btile;
        const uint32_t off = umma::kmajor_offset((uint32_t)n, (uint32_t)(4 * grp));
        *reinterpret_cast<float4*>(bt + off) = hi;
        *reinterpret_cast<float4*>(bt + btile + off) = lo;
      }
      proxy_fence();  // the generic-proxy stores above, before the tensor core's reads
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t sbase = saddr(st);
        const uint32_t bbase = sbase + 2 * NQ * TcStage::kATile;
        auto adesc = [&](int qi, int lohi) {
          return umma::smem_desc(sbase + (uint32_t)(2 * qi + lohi) * TcStage::kATile, umma::kLbo, umma::kSbo);
        };
        auto bdesc = [&](int tab, int lohi) {
          return umma::smem_desc(bbase + (uint32_t)(2 * tab + lohi) * btile, umma::kLbo, umma::kSbo);
        };
        // D_o += A_hi B_hi + A_hi B_lo + A_lo B_hi, for the a terms with C and the b terms with DC
        for (int o = 0; o < 3; ++o) {
          const uint32_t d = tmem + (uint32_t)(o * np);
          const int qa = CURL ? 2 * o : o;             // a_o operand
          const bool hasb = CURL && o < 2;
          const int qb = 2 * o + 1;                    // b_o operand
          uint32_t acc = q > 0 ? 1u : 0u;
          mma_tf32(d, adesc(qa, 0), bdesc(0, 0), idesc, acc);
          mma_tf32(d, adesc(qa, 0), bdesc(0, 1), idesc, 1u);
          mma_tf32(d, adesc(qa, 1), bdesc(0, 0), idesc, 1u);
          if (hasb) {
            mma_tf32(d, adesc(qb, 0), bdesc(1, 0), idesc, 1u);
            mma_tf32(d, adesc(qb, 0), bdesc(1, 1), idesc, 1u);
            mma_tf32(d, adesc(qb, 1), bdesc(1, 0), idesc, 1u);
          }
        }
        mma_commit(&s_bar[sb]);
      }
      ++uses[sb];
    }
    if (!ok) break;
    // all of the tile's MMAs: the last commit covers every earlier one of the issuing thread
    if (nchunks > 0) {
      const int sb = (nchunks - 1) & 1;
      if (!mbar_wait(&s_bar[sb], (uses[sb] - 1) & 1)) {
        if (tid == 0) s_fail = 1;
      }
    }
    __syncthreads();
    if (s_fail) { ok = false; break; }
    tc_fence_after();
    // ---- epilogue: warp w reads its lane quarter (rows 32 (w & 3) ...), half of the 3 Np columns:
    // half 0 from (o, n) = (0, 0), half 1 from (1, Np/2) (Np and 3 Np/2 are multiples of 8)
    {
      const int sp = warp & 3, hf = warp >> 2;
      const int row = 32 * sp + lane;
      const int jr = row >> 1, part = row & 1;
      const int col = s_col[jr];
      const size_t kid = (size_t)s_kid[jr];
      const int ncol = 3 * np, cbeg = hf * (ncol / 2), cend = hf ? ncol : ncol / 2;
      float* kb = reinterpret_cast<float*>(kbuf) + 2 * kid + part;
      const size_t nstride = 2 * (size_t)K;  // floats from coefficient n to n + 1
      int o = hf, n = hf ? np / 2 : 0;
      for (int c8 = cbeg; c8 < cend; c8 += 8) {
        float v[8];
        tmem_ld8(tmem + ((uint32_t)(32 * sp) << 16) + (uint32_t)c8, v);
        if (col >= 0) {
          float* dst = kb + ((size_t)o * N + n) * nstride;
#pragma unroll
          for (int t = 0; t < 8; ++t)
            if (n + t < N) dst[(size_t)t * nstride] = nchunks > 0 ? v[t] : 0.f;
        }
        n += 8;
        if (n >= np) { n -= np; ++o; }
      }
    }
    tc_fence_before();
    __syncthreads();  // the accumulators are read before the next tile's first MMA overwrites them
  }
  if (!ok) {
    if (tid == 0) atomicOr(status, kStatTimeout);
    // one more bounded wait for the MMAs already issued, before the tensor memory is freed
    for (int sb = 0; sb < 2; ++sb)
      if (uses[sb] > 0) mbar_wait(&s_bar[sb], (uses[sb] - 1) & 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, (uint32_t)tcols);
}

}  // namespace

// columns of the tensor-core forward transform's accumulators: three outputs of Np columns
int cheb_tc_np(const Geometry& g) { return (g.nz + 15) / 16 * 16; }

static int tc_tcols(int np) {
  const int need = 3 * np;
  return need <= 32 ? 32 : need <= 64 ? 64 : need <= 128 ? 128 : need <= 256 ? 256 : 512;
}

static size_t tc_smem(const Geometry& g, int np) {
  const bool curl = g.spectral_curl != 0;
  return 2 * (size_t)TcStage::bytes(curl ? 5 : 3, curl ? 2 : 1, np) + 1024;  // two stages, 1 KB alignment slack
}

int cheb_tc_prepare(Plan& p) {
  p.cheb_tc = 0;
  const int np = cheb_tc_np(p.g);
  if (p.precision != DPS_MIXED || p.g.nz > 128 || tc_tcols(np) > 512) return 1;
  if (!allow_smem(cheb_fwd_tc_kernel<true>) || !allow_smem(cheb_fwd_tc_kernel<false>)) return 0;
  int dev = 0, sms = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10) return 1;  // tcgen05: Blackwell data-centre parts only
  p.cheb_tc_grid = sms * (tc_tcols(np) <= 256 ? 2 : 1);
  p.cheb_tc = 1;
  return 1;
}

void launch_cheb_fwd_tc(const Plan& p, int kx0, int w, cudaStream_t s) {
  const Geometry& g = p.g;
  const int np = cheb_tc_np(g);
  const size_t sm = tc_smem(g, np);
  const int64_t tiles = ((int64_t)w * g.ny + kTcWave - 1) / kTcWave;
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, p.cheb_tc_grid));
  const float* ct = reinterpret_cast<const float*>(p.kt.ct);
  const float* dct = reinterpret_cast<const float*>(p.kt.dct);
  const cplx<float>* grid = reinterpret_cast<const cplx<float>*>(p.grid);
  cplx<float>* kbuf = reinterpret_cast<cplx<float>*>(p.kt.kbuf);
  if (g.spectral_curl)
    cheb_fwd_tc_kernel<true><<<blocks, kTcThreads, sm, s>>>(g, ct, dct, p.kt.npad, grid, kbuf, p.zrange, kx0, w, np,
                                                            tc_tcols(np), p.status);
  else
    cheb_fwd_tc_kernel<false><<<blocks, kTcThreads, sm, s>>>(g, ct, dct, p.kt.npad, grid, kbuf, p.zrange, kx0, w, np,
                                                             tc_tcols(np), p.status);
}

}  // namespace dps
