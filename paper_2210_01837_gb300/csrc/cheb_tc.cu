// Chebyshev transforms of the per-wavenumber stage on the 5th-generation tensor cores (mixed
// precision): the forward DCT-I with the half-curl source of the torque route (step 2 of
// Sec. III.D, z part) and the backward step (steps 6-7, z part): inverse DCT-I of the DP
// velocity, the wall correction at the nodes, and the half-curl of Eq. 11.
//
// Both are contractions per wavenumber over one index, with real tables, applied to the real and
// imaginary parts independently.  A block takes 64 wavenumbers as the M = 128 rows of a GEMM (row
// 2j + p: wavenumber j, part p) and runs tcgen05.mma .kind::tf32 over K steps of 8, accumulating
// in tensor memory.  Float accuracy from tf32 operands by the three-product split
// x = x_hi + x_lo, x_hi = tf32(x), x_lo = tf32(x - x_hi):  A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi
// (the dropped A_lo B_lo is 2^-22 relative).
//
//   forward   K = occupied planes c, N = Chebyshev index n (nz rounded up to 16):
//             out_o = C a_o + DC b_o, a_o = f_o + (1/2)(i k x tau)_o, b_x = -tau_y/2, b_y = tau_x/2
//             (DC = (2/H) D C); three accumulators.
//   backward  N = occupied planes (their count rounded up to 16), K = the Chebyshev index n, then
//             (with walls) the node index j:  u_f = IC y_f (f = u, v, w),
//             du = ICD y_u + SD corr_u, dv = ICD y_v + SD corr_v, where corr_f(z_j) is the wall
//             correction at node j (bottom family (cE + cG zeta) e^{-k zeta}, top family
//             (tE + tG xi) e^{-k xi}) and SD = ICD C its spectral derivative (reading B2); five
//             accumulators, [u | du] and [v | dv] each filled by one MMA of N = 2 planes against
//             [IC | ICD] (or [I | SD]), so that A_u and A_v are read once per step.  The epilogue
//             adds corr_f at the output nodes, forms
//             omega = (1/2)(i ky w - dv, du - i kx w, i kx v - i ky u) and scales by 1/(Nx Ny).
//
// The block is persistent over 64-wavenumber tiles and warp-specialised:
//   warps 0-7   producers: load each K step's values from global memory one step ahead (in
//               registers), form and split the step's A operands and store them in the K-major
//               core-matrix layout of one of kStages shared-memory stages, while one thread
//               bulk-copies the step's B operands there from a per-product image (tc_bimage_kernel);
//               each thread fences its stores for the async proxy, and one lane per warp arrives
//               on the stage's `full` barrier (warp-uniform waits and exits, decided by votes);
//   warp 12     MMA issuer: waits for a full stage (and, at a tile's first step, for a free
//               accumulator set), issues the step's MMAs, commits them to the stage's `empty`
//               barrier and, after a tile's last step, to the accumulator set's `full` barrier;
//   warps 8-11  epilogue: wait for a full accumulator set, read it with tcgen05.ld (warp w reads
//               TMEM lanes 32 (w mod 4) ...), write the results, arrive on the set's `empty`
//               barrier.
// Two accumulator sets when their columns fit twice in 512, so a tile's epilogue overlaps the
// next tile's MMAs.  Every barrier wait is bounded (about a second); on expiry the waiting thread
// records DPS_ERR_TIMEOUT in the status word and raises a block-wide stop flag, every role leaves
// its loop, the MMA warp waits once more (bounded) for its last commit, and the tensor memory is
// freed before the block exits.
#include <math.h>

#include <algorithm>

#include "dps_internal.cuh"
#include "umma_desc.h"

namespace dps {
namespace {

constexpr int kTcRows = 128;   // MMA M: 64 wavenumbers x (re, im)
constexpr int kTcK = 8;        // K step (8 tf32 = 32 bytes per operand row)
constexpr int kTcWave = 64;    // wavenumbers per tile
constexpr int kProducers = 256;  // producer threads of one group (8 warps)
// warps of a transform: Spec::kGroups groups of 8 producer warps, then 4 epilogue warps and 1 MMA warp
template <typename Spec> __host__ __device__ constexpr int tc_epi_warp0() { return 8 * Spec::kGroups; }
template <typename Spec> __host__ __device__ constexpr int tc_mma_warp() { return 8 * Spec::kGroups + 4; }
template <typename Spec> __host__ __device__ constexpr int tc_threads() { return 32 * (8 * Spec::kGroups + 5); }
constexpr int kStages = 4;                       // most operand stages (fewer where they do not fit)
constexpr size_t kTcSmemCap = 225 * 1024;        // dynamic shared memory the stages may take
constexpr uint32_t kATile = umma::tile_bytes(kTcRows);  // one A operand of one K step (128 rows x 8)
constexpr long long kWaitCycles = 1ll << 31;     // bounded waits: about one second at 2 GHz

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 2^x by the special-function unit's approximation (ex2.approx; results below the normal range
// flush to zero)
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// tf32 hi part of a float on the integer pipe (no conversion instruction; see tf32_rna_bits)
__device__ __forceinline__ float tf32_rna(float x) { return __uint_as_float(umma::tf32_rna_bits(__float_as_uint(x))); }

// four K-consecutive values of one operand row, split into the hi tile and the lo tile that
// follows it `lo_delta` bytes later
__device__ __forceinline__ void split_store(unsigned char* hi_tile, uint32_t lo_delta, uint32_t off, float a, float b,
                                            float c, float d) {
  const float4 h = make_float4(tf32_rna(a), tf32_rna(b), tf32_rna(c), tf32_rna(d));
  const float4 l = make_float4(tf32_rna(a - h.x), tf32_rna(b - h.y), tf32_rna(c - h.z), tf32_rna(d - h.w));
  *reinterpret_cast<float4*>(hi_tile + off) = h;
  *reinterpret_cast<float4*>(hi_tile + lo_delta + off) = l;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}

// bytes (a multiple of 16, both addresses 16-byte aligned) global -> shared, completing on bar
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// wait for the completion of the phase of the given parity; false after kWaitCycles or once the
// block's stop flag is raised
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, volatile int* stop) {
  const long long t0 = clock64();
  for (;;) {
    if (mbar_test(bar, parity)) return true;
    if (*stop) return false;
    if (clock64() - t0 > kWaitCycles) return false;
  }
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

// D += A_hi B_hi + A_hi B_lo + A_lo B_hi from shared-memory descriptors (A's lo tile follows its
// hi tile by one A tile, B's by b_lo16 16-byte units).  A descriptor's start address is its low
// field in 16-byte units, so the descriptor of an operand `off` bytes further is the stage's
// descriptor plus off >> 4 (shared addresses stay below 256 KB: the field never carries): the
// single issuing thread adds instead of encoding each descriptor anew.
__device__ __forceinline__ void mma3(uint32_t d, uint64_t a_hi, uint64_t b_hi, uint32_t b_lo16, uint32_t idesc,
                                     uint32_t accumulate) {
  constexpr uint64_t kALo16 = kATile >> 4;
  mma_tf32(d, a_hi, b_hi, idesc, accumulate);
  mma_tf32(d, a_hi, b_hi + b_lo16, idesc, 1u);
  mma_tf32(d, a_hi + kALo16, b_hi, idesc, 1u);
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

// 8 consecutive 32-bit columns of this thread's tensor-memory lane, in two steps so that several
// loads share one wait: issue, then wait8 on each issued group (the first wait covers every load
// issued before it; each wait also ties its group's registers, so that no use of them is scheduled
// before the wait)
__device__ __forceinline__ void tmem_issue8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_wait8(uint32_t (&r)[8], float (&v)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
               :
               : "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// wavenumber of tile position j: stored column (-1 past the end), kbuf index, k/2 components, |k|
struct TileK {
  int col;
  int kid;
  float hkx, hky, kk;
};

// pi / Lx, pi / Ly and 1 / (nx ny) in float, formed on the host: in double on the device they take
// divisions on the scarce FP64 pipe at every tile
struct TcScales {
  float hpx, hpy, inv_nxny;
};

// F32: k / 2 as float products with the host's scales (the backward transform: its 20 producer and
// epilogue warps form every tile's wavenumbers, and the double divisions stalled them, 7.08 -> 6.13
// ms on rollers_1m); else in double, rounded once (the forward transform measured faster so, 4.74
// against 4.95 ms)
template <bool F32>
__device__ __forceinline__ TileK tile_k(const Geometry& g, const TcScales& sc, int64_t tile, int j, int kx0, int w) {
  TileK t;
  t.col = -1;
  t.kid = 0;
  t.hkx = t.hky = t.kk = 0.f;
  const int64_t it = tile * kTcWave + j;
  if (it < (int64_t)w * g.ny) {
    const unsigned ii = (unsigned)it;
    const int kyi = (int)(ii / (unsigned)w);
    const int kxi = kx0 + (int)(ii - (unsigned)kyi * (unsigned)w);
    const int nyv = (kyi < (g.ny + 1) / 2) ? kyi : kyi - g.ny;
    t.col = kyi * g.pitch + kxi;
    t.kid = kyi * g.nkx + kxi;
    if (F32) {
      t.hkx = (float)kxi * sc.hpx;
      t.hky = (float)nyv * sc.hpy;
    } else {
      t.hkx = (float)(M_PI * (double)kxi / g.Lx);
      t.hky = (float)(M_PI * (double)nyv / g.Ly);
    }
    t.kk = 2.0f * sqrtf(t.hkx * t.hkx + t.hky * t.hky);
  }
  return t;
}

__device__ __forceinline__ bool is_nyquist(const Geometry& g, int kid) {
  const int kyi = kid / g.nkx, kxi = kid - kyi * g.nkx;
  return ((g.nx % 2 == 0) && kxi == g.nx / 2) || ((g.ny % 2 == 0) && kyi == g.ny / 2);
}

// ---------------------------------------------------------------------------------------------
// forward transform
// ---------------------------------------------------------------------------------------------
template <bool CURL>
struct FwdSpec {
  static constexpr bool kForward = true;
  static constexpr int NQ = CURL ? 5 : 3;  // A operands: a0, b0, a1, b1, a2 (forces only: a0, a1, a2)
  static constexpr int NT = CURL ? 2 : 1;  // B operands: C (and DC)
  static constexpr int NACC = 3;
  static constexpr int NR = CURL ? 4 : 2;  // grid fields a producer thread reads per plane
  static constexpr int kRingDepth = 0;      // loads one step ahead in registers (no staging ring)
  static constexpr int kRingVals = 0;
  static constexpr int kGroups = 1;  // load and store index the producers by threadIdx.x
  struct Args {
    const float* ct;   // [c][npad] C[n][c]
    const float* dct;  // [c][npad] DC[n][c]
    int npad;
    const cplx<float>* grid;
    cplx<float>* kbuf;
  };
  __host__ __device__ static uint32_t stage_bytes(int nmax) { return (uint32_t)(2 * NQ * kATile + 2 * NT * umma::tile_bytes((uint32_t)nmax)); }
  struct Raw {
    cplx<float> v[4][NR];
  };
  // K steps of a tile: the occupied planes in groups of 8
  __host__ __device__ static int nks(const Geometry&, int clo, int chi) {
    return chi >= clo ? (chi - clo + kTcK) / kTcK : 0;
  }
  // producer thread (j, grp, half): wavenumber j, planes 4 grp .. 4 grp + 3 of the step; half 0
  // reads fx, fy, ty, tz (forces only: fx, fy), half 1 reads fz, tx, ty (fz)
  __device__ static void load(const Geometry& g, const Args& a, int clo, int chi, int ks, const TileK& tk, Raw& r) {
    const int tid = threadIdx.x, grp = (tid >> 6) & 1, half = tid >> 7;  // one producer group
    const size_t plane = (size_t)g.ny * g.pitch, fstride = (size_t)g.nz * plane;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int c = clo + ks * kTcK + 4 * grp + cc;
      const bool in = tk.col >= 0 && c <= chi;
      const cplx<float>* p = a.grid + (size_t)(in ? c : 0) * plane + (in ? tk.col : 0);
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        const int f = CURL ? (half == 0 ? (q < 2 ? q : q + 2) : (q < 3 ? q + 2 : 4)) : (half == 0 ? q : 2);
        const bool want = in && (half == 0 || q < (CURL ? 3 : 1));
        r.v[cc][q] = want ? p[(size_t)f * fstride] : mk<float>(0.f, 0.f);
      }
    }
  }
  __device__ static void store(const Geometry& g, const Args& a, int clo, int chi, int ks, const TileK& tk,
                               const Raw& r, unsigned char* st, int np) {
    const int tid = threadIdx.x, j = tid & 63, grp = (tid >> 6) & 1, half = tid >> 7;  // one producer group
    const float hkx = tk.hkx, hky = tk.hky;
    float re[3][4], im[3][4];
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      if (CURL) {
        if (half == 0) {
          const cplx<float> fx = r.v[cc][0], fy = r.v[cc][1], ty = r.v[cc][2], tz = r.v[cc][3];
          // a0 = fx + i ky/2 tz, b0 = -ty/2, a1 = fy - i kx/2 tz
          re[0][cc] = fx.x - hky * tz.y;  im[0][cc] = fx.y + hky * tz.x;
          re[1][cc] = -0.5f * ty.x;       im[1][cc] = -0.5f * ty.y;
          re[2][cc] = fy.x + hkx * tz.y;  im[2][cc] = fy.y - hkx * tz.x;
        } else {
          const cplx<float> fz = r.v[cc][0], tx = r.v[cc][1], ty = r.v[cc][2];
          // b1 = tx/2, a2 = fz + i (kx/2 ty - ky/2 tx)
          const float sx = hkx * ty.x - hky * tx.x, sy = hkx * ty.y - hky * tx.y;
          re[0][cc] = 0.5f * tx.x;  im[0][cc] = 0.5f * tx.y;
          re[1][cc] = fz.x - sy;    im[1][cc] = fz.y + sx;
          re[2][cc] = 0.f;          im[2][cc] = 0.f;
        }
      } else {
        re[0][cc] = r.v[cc][0].x;  im[0][cc] = r.v[cc][0].y;
        re[1][cc] = r.v[cc][1].x;  im[1][cc] = r.v[cc][1].y;
        re[2][cc] = 0.f;           im[2][cc] = 0.f;
      }
    }
    const int nb = CURL ? (half == 0 ? 3 : 2) : (half == 0 ? 2 : 1);
    const int first = half == 0 ? 0 : (CURL ? 3 : 2);
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      if (u >= nb) break;
      unsigned char* ahi = st + (size_t)(2 * (first + u)) * kATile;
      split_store(ahi, kATile, umma::kmajor_offset((uint32_t)(2 * j), (uint32_t)(4 * grp)), re[u][0], re[u][1],
                  re[u][2], re[u][3]);
      split_store(ahi, kATile, umma::kmajor_offset((uint32_t)(2 * j + 1), (uint32_t)(4 * grp)), im[u][0], im[u][1],
                  im[u][2], im[u][3]);
    }
  }
  // B image of step ks, table tab (0: C, 1: DC), row n, plane group kg (4 planes): the tf32 hi/lo
  // split of C[n][c] (DC[n][c]) for c = clo + 8 ks + 4 kg + 0..3, zero outside the occupied planes
  __device__ static void bimage(const Geometry& g, const Args& a, int clo, int chi, int ks, int tab, int n, int kg,
                                unsigned char* step, int np) {
    const float* src = tab == 0 ? a.ct : a.dct;
    float x[4];
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int c = clo + ks * kTcK + 4 * kg + cc;
      x[cc] = (n < g.nz && c <= chi) ? src[(size_t)c * a.npad + n] : 0.f;
    }
    const uint32_t btile = umma::tile_bytes((uint32_t)np);
    split_store(step + (size_t)(2 * tab) * btile, btile, umma::kmajor_offset((uint32_t)n, (uint32_t)(4 * kg)), x[0], x[1],
                x[2], x[3]);
  }
  // sdesc: the descriptor of the stage's first byte
  __device__ static void mma(const Geometry&, uint64_t sdesc, uint32_t tacc, int ks, int np, uint32_t idesc) {
    const uint32_t bt16 = umma::tile_bytes((uint32_t)np) >> 4;
    const uint64_t bbase = sdesc + ((2 * NQ * kATile) >> 4);
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      const uint32_t d = tacc + (uint32_t)(o * np);
      const int qa = CURL ? 2 * o : o;
      mma3(d, sdesc + ((2 * qa * kATile) >> 4), bbase, bt16, idesc, ks > 0 ? 1u : 0u);
      if (CURL && o < 2) mma3(d, sdesc + ((2 * (2 * o + 1) * kATile) >> 4), bbase + 2 * bt16, bt16, idesc, 1u);
    }
  }
  // epilogue thread: TMEM lane `row` (wavenumber row >> 1, part row & 1); out_o[n] -> kbuf (zeros
  // when no plane is occupied)
  __device__ static void epilogue(const Geometry& g, const Args& a, uint32_t tlane, int row, const TileK& tk, int np,
                                  int, int, bool any, float) {
    const int64_t K = (int64_t)g.nkx * g.ny;
    const int N = g.nz, part = row & 1;
    float* kb = reinterpret_cast<float*>(a.kbuf) + 2 * (size_t)tk.kid + part;
    const size_t nstride = 2 * (size_t)K;
    for (int n0 = 0; n0 < np; n0 += 8) {
      float v[3][8];
      if (any) {
        uint32_t r[3][8];
#pragma unroll
        for (int o = 0; o < 3; ++o) tmem_issue8(tlane + (uint32_t)(o * np + n0), r[o]);
#pragma unroll
        for (int o = 0; o < 3; ++o) tmem_wait8(r[o], v[o]);
      }
      if (tk.col < 0) continue;
#pragma unroll
      for (int o = 0; o < 3; ++o) {
        float* dst = kb + ((size_t)o * N + n0) * nstride;
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (n0 + t < N) dst[(size_t)t * nstride] = any ? v[o][t] : 0.f;
      }
    }
  }
};

// ---------------------------------------------------------------------------------------------
// backward transform
// ---------------------------------------------------------------------------------------------
template <int CORR>  // 0 no wall, 1 bottom wall, 2 both walls
struct BwdSpec {
  static constexpr bool kForward = false;
  static constexpr int NQ = 3;  // A operands: y_u, y_v, y_w (node steps: corr_u, corr_v, corr_w)
  static constexpr int NT = 2;  // B operands: IC, ICD (node steps: identity, SD)
  static constexpr int NACC = 5;
  struct Args {
    const float* ict;   // [n][cpad] IC[c][n]
    const float* icdt;  // [n][cpad] ICD[c][n]
    const float* sdt;   // [j][cpad] SD[c][j]
    int cpad;
    const float* zeta;  // [nz] z_c - zmin
    const cplx<float>* kbuf;
    const cplx<float>* kaux;
    cplx<float>* grid;
  };
  __host__ __device__ static uint32_t stage_bytes(int nmax) {
    return (uint32_t)(2 * NQ * kATile + 2 * NT * umma::tile_bytes((uint32_t)nmax));
  }
  // coefficient step: v[cc][q] = y_f[n], n = 8 ks + 4 grp + cc (half 0: f = u, v; half 1: f = w);
  // node step: v[q][fi] = amplitude q (cE, cG, tE, tG) of field f (half 0: u, v; half 1: w)
  struct Raw {
    cplx<float> v[4][2];
  };
  // two producer groups take alternate K steps; each stages its steps' values with cp.async
  // kRingDepth - 1 of its own steps ahead into its ring in shared memory (value e of group thread t
  // of a slot at slot[e * kProducers + t])
  static constexpr int kGroups = 2;
  static constexpr int kRingDepth = 2;
  static constexpr int kRingVals = 8;
  __host__ __device__ static int ncoef(const Geometry& g) { return (g.nz + kTcK - 1) / kTcK; }
  __host__ __device__ static int nks(const Geometry& g, int, int) { return ncoef(g) * (CORR ? 2 : 1); }
  // the values `load` would read, copied asynchronously into ring slot `slot` (zeros where load
  // reads none); completes in the calling thread's current cp.async group
  __device__ static void load_async(const Geometry& g, const Args& a, int ks, const TileK& tk, cplx<float>* slot) {
    const int tid = threadIdx.x & (kProducers - 1), grp = (tid >> 6) & 1, half = tid >> 7;
    const int64_t K = (int64_t)g.nkx * g.ny;
    const int N = g.nz;
    const bool ok = tk.col >= 0;
    if (ks < ncoef(g)) {
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int n = ks * kTcK + 4 * grp + cc;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int f = half == 0 ? q : 2;
          const bool want = ok && n < N && (half == 0 || q == 0);
          cplx<float>* dst = slot + (cc * 2 + q) * kProducers + tid;
          if (want) cp_async8(dst, a.kbuf + ((size_t)f * N + n) * K + tk.kid);
          else *dst = mk<float>(0.f, 0.f);
        }
      }
    } else {
      const bool amp = ok && tk.kid > 0 && !is_nyquist(g, tk.kid);
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int fi = 0; fi < 2; ++fi) {
          const int f = half == 0 ? fi : 2;
          const bool want = amp && (q < 2 || CORR == 2) && (half == 0 || fi == 0);
          cplx<float>* dst = slot + (q * 2 + fi) * kProducers + tid;
          if (want) cp_async8(dst, a.kaux + (size_t)(4 * f + q) * K + tk.kid);
          else *dst = mk<float>(0.f, 0.f);
        }
    }
  }
  __device__ static void from_ring(const cplx<float>* slot, Raw& r) {
    const int tid = threadIdx.x & (kProducers - 1);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int q = 0; q < 2; ++q) r.v[i][q] = slot[(i * 2 + q) * kProducers + tid];
  }
  __device__ static void load(const Geometry& g, const Args& a, int, int, int ks, const TileK& tk, Raw& r) {
    const int tid = threadIdx.x & (kProducers - 1), grp = (tid >> 6) & 1, half = tid >> 7;
    const int64_t K = (int64_t)g.nkx * g.ny;
    const int N = g.nz;
    const bool ok = tk.col >= 0;
    if (ks < ncoef(g)) {
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int n = ks * kTcK + 4 * grp + cc;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int f = half == 0 ? q : 2;
          const bool want = ok && n < N && (half == 0 || q == 0);
          r.v[cc][q] = want ? a.kbuf[((size_t)f * N + n) * K + tk.kid] : mk<float>(0.f, 0.f);
        }
      }
    } else {
      const bool amp = ok && tk.kid > 0 && !is_nyquist(g, tk.kid);
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int fi = 0; fi < 2; ++fi) {
          const int f = half == 0 ? fi : 2;
          const bool want = amp && (q < 2 || CORR == 2) && (half == 0 || fi == 0);
          r.v[q][fi] = want ? a.kaux[(size_t)(4 * f + q) * K + tk.kid] : mk<float>(0.f, 0.f);
        }
    }
  }
  __device__ static void store(const Geometry& g, const Args& a, int, int, int ks, const TileK& tk, const Raw& r,
                               unsigned char* st, int) {
    const int tid = threadIdx.x & (kProducers - 1), j = tid & 63, grp = (tid >> 6) & 1, half = tid >> 7;
    const int N = g.nz;
    const uint32_t orow = umma::kmajor_offset((uint32_t)(2 * j), (uint32_t)(4 * grp));
    const uint32_t orow1 = umma::kmajor_offset((uint32_t)(2 * j + 1), (uint32_t)(4 * grp));
    float re[2][4], im[2][4];
    if (ks < ncoef(g)) {
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          re[q][cc] = r.v[cc][q].x;
          im[q][cc] = r.v[cc][q].y;
        }
    } else {
      // corr_f at the step's nodes: (cE + cG zeta) e^{-k zeta} (+ (tE + tG xi) e^{-k xi}), the
      // exponentials as 2^(-k log2(e) zeta) on the special-function unit (relative error about
      // 2^-22, and |k log2(e) zeta| 2^-24 from the rounded argument: float level)
      const int j0 = (ks - ncoef(g)) * kTcK + 4 * grp;
      const float kl = -tk.kk * 1.4426950408889634f;  // -k log2(e)
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int jn = j0 + cc;
        float z = 0.f, eb = 0.f, xi = 0.f, et = 0.f;
        if (jn < N) {
          z = a.zeta[jn];
          eb = ex2_approx(kl * z);
          if (CORR == 2) {
            xi = a.zeta[N - 1 - jn];
            et = ex2_approx(kl * xi);
          }
        }
#pragma unroll
        for (int fi = 0; fi < 2; ++fi) {
          float vx = (r.v[0][fi].x + r.v[1][fi].x * z) * eb, vy = (r.v[0][fi].y + r.v[1][fi].y * z) * eb;
          if (CORR == 2) {
            vx += (r.v[2][fi].x + r.v[3][fi].x * xi) * et;
            vy += (r.v[2][fi].y + r.v[3][fi].y * xi) * et;
          }
          re[fi][cc] = vx;
          im[fi][cc] = vy;
        }
      }
    }
    // A operands: u, v (half 0) or w (half 1)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (half == 1 && q == 1) break;
      unsigned char* ahi = st + (size_t)(2 * (half == 0 ? q : 2)) * kATile;
      split_store(ahi, kATile, orow, re[q][0], re[q][1], re[q][2], re[q][3]);
      split_store(ahi, kATile, orow1, im[q][0], im[q][1], im[q][2], im[q][3]);
    }
  }
  // B image of step ks, table tab, row p (plane clo + p), index group kg: coefficient steps tab 0
  // IC[c][n], tab 1 ICD[c][n]; node steps tab 0 the identity (c = j), tab 1 SD[c][j]; zero outside
  // the occupied planes and past the last index
  __device__ static void bimage(const Geometry& g, const Args& a, int clo, int chi, int ks, int tab, int p, int kg,
                                unsigned char* step, int nq) {
    const int N = g.nz, nc = ncoef(g);
    const int c = clo + p;
    float x[4];
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int idx = (ks < nc ? ks : ks - nc) * kTcK + 4 * kg + cc;
      float v = 0.f;
      if (c <= chi && idx < N) {
        if (ks < nc) v = (tab == 0 ? a.ict : a.icdt)[(size_t)idx * a.cpad + c];
        else v = tab == 0 ? (idx == c ? 1.f : 0.f) : a.sdt[(size_t)idx * a.cpad + c];
      }
      x[cc] = v;
    }
    // [B0; B1] as one operand of 2 nq rows (hi), its lo part 2 btile further
    const uint32_t btile = umma::tile_bytes((uint32_t)nq);
    split_store(step, 2 * btile, umma::kmajor_offset((uint32_t)(tab * nq + p), (uint32_t)(4 * kg)), x[0], x[1], x[2],
                x[3]);
  }
  // every step: [u | du] += A_u [B0 | B1], [v | dv] += A_v [B0 | B1] (N = 2 nq), w += A_w B0
  // sdesc: the descriptor of the stage's first byte
  __device__ static void mma(const Geometry&, uint64_t sdesc, uint32_t tacc, int ks, int nq, uint32_t idesc) {
    const uint32_t lo16 = (2 * umma::tile_bytes((uint32_t)nq)) >> 4;  // the lo block of [B0; B1]
    const uint64_t b0 = sdesc + ((2 * NQ * kATile) >> 4);
    const uint32_t acc = ks > 0 ? 1u : 0u;
    const uint32_t idesc2 = idesc + (((uint32_t)nq >> 3) << 17);  // N = 2 nq (the N >> 3 field doubled)
    const uint64_t au = sdesc, av = sdesc + ((2 * kATile) >> 4), aw = sdesc + ((4 * kATile) >> 4);
    mma3(tacc + 0 * nq, au, b0, lo16, idesc2, acc);  // u, du
    mma3(tacc + 2 * nq, av, b0, lo16, idesc2, acc);  // v, dv
    mma3(tacc + 4 * nq, aw, b0, lo16, idesc, acc);   // w
  }
  // epilogue thread: TMEM lane `row` = (wavenumber row >> 1, part row & 1); lanes 2j and 2j + 1 pair
  // up for the products with i
  __device__ static void epilogue(const Geometry& g, const Args& a, uint32_t tlane, int row, const TileK& tk, int nq,
                                  int clo, int chi, bool, float inv_nxny) {
    const int part = row & 1;
    const bool nyq = tk.col >= 0 && is_nyquist(g, tk.kid);
    const float scale = nyq ? 0.f : inv_nxny;
    const size_t plane = (size_t)g.ny * g.pitch, fstride = (size_t)g.nz * plane;
    float* gr = reinterpret_cast<float*>(a.grid) + 2 * (size_t)(tk.col >= 0 ? tk.col : 0) + part;
    const float sgn = part ? 1.f : -1.f;  // (i x) of this part: re -> -x.im, im -> +x.re
    const float hx = tk.hkx * scale, hy = tk.hky * scale, hs = 0.5f * scale;
    for (int p0 = 0; p0 < nq; p0 += 8) {
      float u[8], v[8], w[8], du[8], dv[8];
      uint32_t r[5][8];
#pragma unroll
      for (int q = 0; q < 5; ++q) tmem_issue8(tlane + (uint32_t)(q * nq + p0), r[q]);
      tmem_wait8(r[0], u);
      tmem_wait8(r[1], du);
      tmem_wait8(r[2], v);
      tmem_wait8(r[3], dv);
      tmem_wait8(r[4], w);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int c = clo + p0 + t;
        // the other part of u, v, w (partner lane); (i x) of this part = sgn x(other part)
        const float iu = sgn * __shfl_xor_sync(0xffffffffu, u[t], 1);
        const float iv = sgn * __shfl_xor_sync(0xffffffffu, v[t], 1);
        const float iw = sgn * __shfl_xor_sync(0xffffffffu, w[t], 1);
        if (tk.col >= 0 && c <= chi) {
          // omega = 1/2 (i ky w - dv, du - i kx w, i kx v - i ky u), all scaled by 1/(Nx Ny)
          float* o = gr + 2 * (size_t)c * plane;
          o[0] = u[t] * scale;
          o[2 * fstride] = v[t] * scale;
          o[4 * fstride] = w[t] * scale;
          o[6 * fstride] = hy * iw - hs * dv[t];
          o[8 * fstride] = hs * du[t] - hx * iw;
          o[10 * fstride] = hx * iv - hy * iu;
        }
      }
    }
  }
};

// ---------------------------------------------------------------------------------------------
// the pipeline
// ---------------------------------------------------------------------------------------------
struct TcShared {
  uint64_t full[kStages], empty[kStages];
  uint64_t acc_full[2], acc_empty[2];
  uint32_t tmem;
  int stop;
};

// GEMM N of a transform: forward the Chebyshev index, backward the occupied planes (their count),
// rounded up to 16 (at least 16)
template <typename Spec>
__host__ __device__ inline int tc_nn(const Geometry& g, int clo, int chi) {
  const int nmax = (g.nz + 15) / 16 * 16;
  const int nocc = chi >= clo ? chi - clo + 1 : 0;
  const int nq = (nocc + 15) / 16 * 16;
  return Spec::kForward ? nmax : (nq < 16 ? 16 : nq);
}

// The backward transform's output planes in `nparts` parts (one launch each) when five
// accumulators of all of them would not fit the 512 tensor-memory columns: part `part` of the
// occupied range [clo, chi], parts of a multiple of 16 planes; an empty part has lo > hi.
__host__ __device__ inline void tc_part(int& clo, int& chi, int part, int nparts) {
  if (nparts <= 1) return;
  const int nocc = chi >= clo ? chi - clo + 1 : 0;
  const int ph = ((nocc + nparts - 1) / nparts + 15) / 16 * 16;
  const int lo = clo + part * ph;
  chi = min(chi, lo + ph - 1);
  clo = lo;
}

// The B operands of every K step of a product, tf32-split and laid out as in a stage, so that the
// pipeline copies them with one bulk copy per step: image[ks][tab][hi, lo][nn rows x 8]
template <typename Spec>
__global__ void tc_bimage_kernel(Geometry g, typename Spec::Args a, const int* __restrict__ zrange,
                                 unsigned char* __restrict__ img, int part, int nparts) {
  int clo = zrange[0], chi = zrange[1];
  tc_part(clo, chi, part, nparts);
  if (chi < clo && nparts > 1) return;  // an empty part
  const int nn = tc_nn<Spec>(g, clo, chi);
  const int nks = Spec::nks(g, clo, chi);
  const uint32_t step = (uint32_t)(2 * Spec::NT * umma::tile_bytes((uint32_t)nn));
  const int items = nks * Spec::NT * nn * 2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < items; i += gridDim.x * blockDim.x) {
    const int kg = i & 1, r = (i >> 1) % nn, rest = (i >> 1) / nn;
    const int tab = rest % Spec::NT, ks = rest / Spec::NT;
    Spec::bimage(g, a, clo, chi, ks, tab, r, kg, img + (size_t)ks * step, nn);
  }
}

template <typename Spec>
__global__ void __launch_bounds__(tc_threads<Spec>(), 1) cheb_tc_kernel(Geometry g, typename Spec::Args a, TcScales sc,
                                                                const unsigned char* __restrict__ bimg,
                                                                const int* __restrict__ zrange, int kx0, int w,
                                                                int* __restrict__ status, int inject, int part,
                                                                int nparts) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ TcShared sh;
  __shared__ float s_zeta[128];  // backward: the node heights, read by every node step
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int clo = zrange[0], chi = zrange[1];
  tc_part(clo, chi, part, nparts);  // the backward transform's output planes of this launch
  if (chi < clo && nparts > 1) return;  // an empty part (uniform over the grid)
  const int64_t ntiles = ((int64_t)w * g.ny + kTcWave - 1) / kTcWave;
  const int nmax = (g.nz + 15) / 16 * 16;  // the stage layout is sized for this
  const int nn = tc_nn<Spec>(g, clo, chi);
  const uint32_t bbytes = (uint32_t)(2 * Spec::NT * umma::tile_bytes((uint32_t)nn));  // B operands of one step
  const int cols = Spec::NACC * nn;
  const int nbuf = 2 * cols <= 512 ? 2 : 1;
  const int need = nbuf * cols;
  const uint32_t tcols = need <= 32 ? 32 : need <= 64 ? 64 : need <= 128 ? 128 : need <= 256 ? 256 : 512;
  const uint32_t stage_bytes = Spec::stage_bytes(nmax);
  uint32_t dyn;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
  constexpr uint32_t kRingBytes = (uint32_t)(Spec::kGroups * Spec::kRingDepth * Spec::kRingVals * kProducers * 8);
  constexpr int kEpiWarp0 = tc_epi_warp0<Spec>(), kMmaWarp = tc_mma_warp<Spec>();
  const int nst = min(kStages, (int)((dyn - 1024u - kRingBytes) / stage_bytes));  // operand stages launched with
  const int nks = Spec::nks(g, clo, chi);
  const uint32_t idesc = umma::idesc_tf32(kTcRows, (uint32_t)nn);
  volatile int* stop = &sh.stop;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sh.full[s], kProducers / 32 + 1);  // a lane of each producer warp, and the B copy's arming
      mbar_init(&sh.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.acc_full[b], 1);
      mbar_init(&sh.acc_empty[b], 128);
    }
    sh.stop = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&sh.tmem)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if constexpr (!Spec::kForward) {
    for (int i = tid; i < g.nz; i += tc_threads<Spec>()) s_zeta[i] = a.zeta[i];  // nz <= 128 here
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if constexpr (!Spec::kForward) a.zeta = s_zeta;
  const uint32_t tmem = sh.tmem;
  auto fail = [&]() {
    if (!*stop) {
      sh.stop = 1;
      atomicOr(status, kStatTimeout);
    }
  };
  if constexpr (Spec::kRingDepth > 0) {
    if (warp < kEpiWarp0) {
      // ---- producers, staging through the ring --------------------------------------------
      // group gp takes the block's K steps q = gp, gp + G, gp + 2 G, ... (q counts the steps of the
      // block's tiles in order, nks per tile; step q fills operand stage q mod nst, which the MMA
      // warp consumes in the order of q), staging its own steps' values D - 1 of them ahead
      constexpr int D = Spec::kRingDepth, G = Spec::kGroups;
      const int gp = warp >> 3, gtid = tid & (kProducers - 1);
      cplx<float>* ring = reinterpret_cast<cplx<float>*>(smraw + (size_t)nst * stage_bytes) +
                          (size_t)gp * D * Spec::kRingVals * kProducers;
      auto slot = [&](int i) { return ring + (size_t)i * Spec::kRingVals * kProducers; };
      auto advance = [&](int64_t& tile, int& ks, int by) {  // (tile, step) of the step `by` (<= G) later
        ks += by;
        if (ks >= nks) {
          ks -= nks;
          tile += gridDim.x;
          if (ks >= nks) {  // nks < G: one step per tile
            ks -= nks;
            tile += gridDim.x;
          }
        }
      };
      int64_t lt = blockIdx.x, st_tile = blockIdx.x;  // tiles of the next step to stage / to store
      int lks = 0, sks = 0;
      if (nks > 0) {
        advance(lt, lks, gp);
        advance(st_tile, sks, gp);
      }
      if (st_tile < ntiles && nks > 0) {
        TileK ltk = tile_k<!Spec::kForward>(g, sc, lt, tid & 63, kx0, w), stk = ltk;
        // one cp.async group per step (an empty one past the last step), so that waiting for all
        // but the D - 1 newest groups completes the current step's
        auto stage_next = [&](int i) {
          if (lt < ntiles) Spec::load_async(g, a, lks, ltk, slot(i));
          cp_commit();
          const int64_t t0 = lt;
          advance(lt, lks, G);
          if (lt != t0 && lt < ntiles) ltk = tile_k<!Spec::kForward>(g, sc, lt, tid & 63, kx0, w);
        };
        for (int i = 0; i < D - 1; ++i) stage_next(i);
        int s = gp, rs = 0, ws = D - 1;  // operand stage (G <= nst); ring slots to read / to fill
        unsigned ph = 0;
        for (;;) {
          // the loads D - 1 own steps ahead go out first (their ring slot was read in the previous
          // step), before the wait for a free operand stage
          stage_next(ws);
          ws = ws + 1 == D ? 0 : ws + 1;
          // warp-uniform decisions: the warp's lanes arrive once, together (see below)
          if (!__all_sync(0xffffffffu, mbar_wait(&sh.empty[s], ph ^ 1, stop))) { fail(); break; }
          unsigned char* st = smraw + (size_t)s * stage_bytes;
          if (gtid == 0) {
            mbar_arrive_tx(&sh.full[s], bbytes);
            bulk_copy(st + 2 * Spec::NQ * kATile, bimg + (size_t)sks * bbytes, bbytes, &sh.full[s]);
          }
          asm volatile("cp.async.wait_group %0;\n" ::"n"(D - 1) : "memory");
          typename Spec::Raw cur;
          Spec::from_ring(slot(rs), cur);
          rs = rs + 1 == D ? 0 : rs + 1;
          Spec::store(g, a, clo, chi, sks, stk, cur, st, nn);
          proxy_fence();
          __syncwarp();  // the warp's stores, each fenced by its thread, before its one arrival
          if (lane == 0) mbar_arrive(&sh.full[s]);
          s += G;
          if (s >= nst) {
            s -= nst;
            ph ^= 1u;
          }
          const int64_t t0 = st_tile;
          advance(st_tile, sks, G);
          if (st_tile != t0) {
            if (__any_sync(0xffffffffu, st_tile >= ntiles || *stop)) break;
            stk = tile_k<!Spec::kForward>(g, sc, st_tile, tid & 63, kx0, w);
          }
        }
        cp_wait_all();  // no copy into the ring outlives the loop
      }
    }
  }
  if (Spec::kRingDepth > 0 && warp < kEpiWarp0) {
    // the producers above
  } else if (warp < kEpiWarp0) {
    // ---- producers ------------------------------------------------------------------------
    int s = 0;        // stage of the next K step
    unsigned ph = 0;  // its use parity (the stage ring's pass)
    typename Spec::Raw raw;
    int64_t tile = blockIdx.x;
    if (tile < ntiles && nks > 0) {
      TileK tk = tile_k<!Spec::kForward>(g, sc, tile, tid & 63, kx0, w);
      Spec::load(g, a, clo, chi, 0, tk, raw);
      for (;;) {
        for (int ks = 0; ks < nks; ++ks) {
          // warp-uniform decisions: the warp's lanes arrive once, together (see below)
          if (!__all_sync(0xffffffffu, mbar_wait(&sh.empty[s], ph ^ 1, stop))) { fail(); break; }
          unsigned char* st = smraw + (size_t)s * stage_bytes;
          const typename Spec::Raw cur = raw;
          // the next step's loads, issued before this step's stores
          const bool last = ks + 1 == nks;
          const int64_t ntile = last ? tile + gridDim.x : tile;
          const TileK ntk = last ? tile_k<!Spec::kForward>(g, sc, ntile, tid & 63, kx0, w) : tk;
          // the step's B operands: one bulk copy from the image, completing on the stage barrier
          if (tid == 0) {
            mbar_arrive_tx(&sh.full[s], bbytes);
            bulk_copy(st + 2 * Spec::NQ * kATile, bimg + (size_t)ks * bbytes, bbytes, &sh.full[s]);
          }
          if (ntile < ntiles) Spec::load(g, a, clo, chi, last ? 0 : ks + 1, ntk, raw);
          Spec::store(g, a, clo, chi, ks, tk, cur, st, nn);
          proxy_fence();
          __syncwarp();  // the warp's stores, each fenced by its thread, before its one arrival
          if (lane == 0) mbar_arrive(&sh.full[s]);
          if (last) tk = ntk;
          if (++s == nst) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (__any_sync(0xffffffffu, *stop != 0)) break;
        tile += gridDim.x;
        if (tile >= ntiles) break;
      }
    }
  } else if (warp == kMmaWarp) {
    // ---- MMA issuer -----------------------------------------------------------------------
    unsigned it = 0, t = 0;
    const uint64_t sdesc0 = umma::smem_desc(saddr(smraw), umma::kLbo, umma::kSbo);  // stage 0
    int s = 0, ls = 0;           // stage of the next K step, of the last one issued
    unsigned ph = 0, lph = 0;    // their use parities
    for (int64_t tile = blockIdx.x; tile < ntiles && nks > 0 && !*stop; tile += gridDim.x, ++t) {
      const int b = nbuf == 2 ? (int)(t & 1) : 0;
      const unsigned use = nbuf == 2 ? t >> 1 : t;  // earlier uses of this accumulator set
      if (!mbar_wait(&sh.acc_empty[b], (use & 1) ^ 1, stop)) { fail(); break; }
      tc_fence_after();
      const uint32_t tacc = tmem + (uint32_t)(b * cols);
      bool ok = true;
      for (int ks = 0; ks < nks; ++ks, ++it) {
        if (!mbar_wait(&sh.full[s], ph, stop)) { fail(); ok = false; break; }
        tc_fence_after();
        ls = s;
        lph = ph;
        if (++s == nst) {
          s = 0;
          ph ^= 1u;
        }
        if (inject) continue;  // failure injection: no MMAs and no completion signals
        if (lane == 0) {
          Spec::mma(g, sdesc0 + (((uint32_t)ls * stage_bytes) >> 4), tacc, ks, nn, idesc);
          mma_commit(&sh.empty[ls]);  // the stage is free once these MMAs have read it
          if (ks + 1 == nks) mma_commit(&sh.acc_full[b]);
        }
        __syncwarp();
      }
      if (!ok) break;
    }
    // a stop: wait (bounded) for the MMAs already issued before the tensor memory is freed
    if (*stop && it > 0 && !inject) {
      const long long t0 = clock64();
      while (!mbar_test(&sh.empty[ls], lph) && clock64() - t0 < kWaitCycles) {
      }
    }
  } else {
    // ---- epilogue ---------------------------------------------------------------------------
    const int row = 32 * (warp & 3) + lane;
    const uint32_t tlane = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    unsigned t = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++t) {
      const TileK tk = tile_k<!Spec::kForward>(g, sc, tile, row >> 1, kx0, w);
      if (nks == 0) {  // forward with no occupied plane: zero coefficients
        Spec::epilogue(g, a, tlane, row, tk, nn, clo, chi, false, sc.inv_nxny);
        continue;
      }
      const int b = nbuf == 2 ? (int)(t & 1) : 0;
      const unsigned use = nbuf == 2 ? t >> 1 : t;
      if (!mbar_wait(&sh.acc_full[b], use & 1, stop)) { fail(); break; }
      tc_fence_after();
      Spec::epilogue(g, a, tlane + (uint32_t)(b * cols), row, tk, nn, clo, chi, true, sc.inv_nxny);
      tc_fence_before();
      mbar_arrive(&sh.acc_empty[b]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
  }
}

template <typename Spec>
size_t tc_smem(const Geometry& g) {
  // as many operand stages as fit (at most kStages); 0 when fewer than two fit
  const size_t sb = Spec::stage_bytes((g.nz + 15) / 16 * 16);
  const size_t ring = (size_t)Spec::kGroups * Spec::kRingDepth * Spec::kRingVals * kProducers * 8;
  const size_t n = std::min<size_t>(kStages, (kTcSmemCap - 1024 - ring) / sb);
  return n >= 2 ? n * sb + ring + 1024 : 0;
}

template <typename Spec>
void launch_tc(const Plan& p, const typename Spec::Args& a, unsigned char* img, int kx0, int w, cudaStream_t s,
               int inject = 0, int nparts = 1) {
  const int64_t tiles = ((int64_t)w * p.g.ny + kTcWave - 1) / kTcWave;
  const TcScales sc{(float)(M_PI / p.g.Lx), (float)(M_PI / p.g.Ly), (float)(1.0 / ((double)p.g.nx * p.g.ny))};
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, p.cheb_tc_grid));
  for (int part = 0; part < nparts; ++part) {
    tc_bimage_kernel<Spec><<<64, 256, 0, s>>>(p.g, a, p.zrange, img, part, nparts);
    cheb_tc_kernel<Spec><<<blocks, tc_threads<Spec>(), tc_smem<Spec>(p.g), s>>>(p.g, a, sc, img, p.zrange, kx0, w, p.status,
                                                                        inject, part, nparts);
  }
}

}  // namespace

int cheb_tc_np(const Geometry& g) { return (g.nz + 15) / 16 * 16; }

size_t cheb_tc_image_bytes(const Geometry& g, bool backward) {
  const size_t nmax = (size_t)cheb_tc_np(g), ksteps = (size_t)(g.nz + kTcK - 1) / kTcK;
  return (backward ? 2 * ksteps : ksteps) * 2 * 2 * umma::tile_bytes((uint32_t)nmax);
}

int cheb_tc_prepare(Plan& p) {
  p.cheb_tc = 0;
  p.cheb_tc_bwd = 0;
  if (p.precision != DPS_MIXED || p.g.nz > 128) return 1;
  int dev = 0, sms = 0, major = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (major != 10) return 1;  // tcgen05: Blackwell data-centre parts only
  if (!allow_smem(cheb_tc_kernel<FwdSpec<true>>) || !allow_smem(cheb_tc_kernel<FwdSpec<false>>) ||
      !allow_smem(cheb_tc_kernel<BwdSpec<0>>) || !allow_smem(cheb_tc_kernel<BwdSpec<1>>) ||
      !allow_smem(cheb_tc_kernel<BwdSpec<2>>))
    return 0;
  p.cheb_tc_grid = sms;
  const size_t sf = tc_smem<FwdSpec<true>>(p.g), sb = tc_smem<BwdSpec<2>>(p.g);
  if (sf > 0 && sf + 1024 <= (size_t)optin) p.cheb_tc = 1;
  // backward: five accumulators of the occupied planes (rounded up to 16) must fit 512 columns;
  // beyond 96 nodes the planes go in two launches of at most 64 each
  if (p.g.spectral_curl && sb > 0 && sb + 1024 <= (size_t)optin) {
    p.cheb_tc_bwd = 1;
    p.cheb_tc_bwd_parts = 5 * cheb_tc_np(p.g) <= 512 ? 1 : 2;
  }
  return 1;
}

void launch_cheb_fwd_tc(const Plan& p, int kx0, int w, cudaStream_t s) {
  const Geometry& g = p.g;
  if (g.spectral_curl) {
    const FwdSpec<true>::Args a{reinterpret_cast<const float*>(p.kt.ct), reinterpret_cast<const float*>(p.kt.dct),
                                p.kt.npad, reinterpret_cast<const cplx<float>*>(p.grid),
                                reinterpret_cast<cplx<float>*>(p.kt.kbuf)};
    launch_tc<FwdSpec<true>>(p, a, p.kt.bimg_f, kx0, w, s, p.inject == 1 ? 1 : 0);
  } else {
    const FwdSpec<false>::Args a{reinterpret_cast<const float*>(p.kt.ct), reinterpret_cast<const float*>(p.kt.dct),
                                 p.kt.npad, reinterpret_cast<const cplx<float>*>(p.grid),
                                 reinterpret_cast<cplx<float>*>(p.kt.kbuf)};
    launch_tc<FwdSpec<false>>(p, a, p.kt.bimg_f, kx0, w, s, p.inject == 1 ? 1 : 0);
  }
}

void launch_cheb_bwd_tc(const Plan& p, int kx0, int w, cudaStream_t s) {
  const Geometry& g = p.g;
  const float* ict = reinterpret_cast<const float*>(p.kt.ict);
  const float* icdt = reinterpret_cast<const float*>(p.kt.icdt);
  const float* sdt = reinterpret_cast<const float*>(p.kt.sdt);
  const float* zeta = reinterpret_cast<const float*>(p.tab.zeta);
  const cplx<float>* kbuf = reinterpret_cast<const cplx<float>*>(p.kt.kbuf);
  const cplx<float>* kaux = reinterpret_cast<const cplx<float>*>(p.kt.kaux);
  cplx<float>* grid = reinterpret_cast<cplx<float>*>(p.grid);
  if (g.mode == DPS_FREE)
    launch_tc<BwdSpec<0>>(p, BwdSpec<0>::Args{ict, icdt, sdt, p.kt.cpad, zeta, kbuf, kaux, grid}, p.kt.bimg_b, kx0, w,
                           s, 0, p.cheb_tc_bwd_parts);
  else if (g.mode == DPS_BOTTOM_WALL)
    launch_tc<BwdSpec<1>>(p, BwdSpec<1>::Args{ict, icdt, sdt, p.kt.cpad, zeta, kbuf, kaux, grid}, p.kt.bimg_b, kx0, w,
                           s, 0, p.cheb_tc_bwd_parts);
  else
    launch_tc<BwdSpec<2>>(p, BwdSpec<2>::Args{ict, icdt, sdt, p.kt.cpad, zeta, kbuf, kaux, grid}, p.kt.bimg_b, kx0, w,
                           s, 0, p.cheb_tc_bwd_parts);
}

}  // namespace dps
