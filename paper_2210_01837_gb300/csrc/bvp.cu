// Per-wavenumber stage of the doubly-periodic Stokes solve (steps 2-7 of Sec. III.D, z part).
//
// Three kernels, each shaped for the pipe it needs, with one thread per (kx, ky) of the half
// spectrum and k-contiguous (coalesced) layouts throughout:
//
//   fwd_kernel   (transform precision T)  Chebyshev coefficients of the three force components by
//                DCT-I of the occupied planes, with the half-curl of the torque field added in
//                Fourier-Chebyshev space (Eq. 7); written to the coefficient buffer kbuf[3][N][K].
//   solve_kernel (FP64)                   DP pressure BVP (Eqs. 15, 17), DP velocity BVPs
//                (Eqs. 18, 22, 24) with the shared factorisation, boundary values of the DP velocity
//                by direct summation and the wall-correction amplitudes (bottom wall Eqs. 41-44;
//                slit Eqs. A4-A10 with zero slip, in closed form); k = 0 (Sec. III.C, Eq. A12).
//                Writes the DP velocity coefficients over kbuf and the amplitudes to kaux.
//   bwd_kernel   (transform precision T)  node values on the occupied planes: inverse DCT-I of the DP
//                coefficients plus the correction evaluated at the nodes (step 6), and, with torques,
//                the half-curl (Eq. 11) from the Chebyshev derivative of the summed interpolant; times
//                1/(Nx Ny) for the inverse xy transform.  Nyquist modes are set to zero.
//
// The FP64 pipe of this GPU is ~1/58 of the FP32 rate and also executes float<->double conversions,
// so the solve kernel converts with integer bit operations (exact widening; narrowing by
// truncation, 2^-23 relative) and forms right-hand sides in the transform precision; the banded
// sweeps, the factorisation, the boundary rows and the correction amplitudes are FP64.
//
// BVP discretisation (the paper defers it to Greengard's spectral integration): s in [-1, 1],
// y = trunc_N(B B c) + a0 T0 + a1 T1 with c the coefficients of y_ss; rows
// (2/H)^2 c_n - k^2 y_n = r_n, n = 0..N-1, plus two boundary rows.  B B couples c_{n-2}, c_n,
// c_{n+2} only (coefficients l_n, d_n, u_n), so the system splits into an even and an odd
// tridiagonal system, each bordered by one unknown (a0 or a1, row 0 or 1) and by one dense
// boundary row; the Dirichlet-to-Neumann rows combine into one row per parity.  Each parity is
// eliminated from the last row down (c_n = s_n - t_n c_{n-2}) while the boundary row is folded,
// leaving a 2x2 system for (c_par, a_par); the rows are diagonally dominant, so no pivoting.
#include <math.h>

#include <algorithm>

#include "dps_internal.cuh"

namespace dps {

namespace {

// ---------------------------------------------------------------------------------------------
// conversions on the integer pipe
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double f2d(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  if (e == 0u) return 0.0;  // zero (float subnormals flush to zero)
  const unsigned m = b & 0x7fffffu;
  const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | (m >> 3);
  return __hiloint2double((int)hi, (int)(m << 29));
}

__device__ __forceinline__ float d2f(double d) { return narrow_bits(d); }

// 1/d for the pivots of the factorisation (|d| well inside the float range) by Newton-Raphson from a
// float seed: x0 = approximate float reciprocal of the narrowed d (relative error about 2^-22),
// then x <- x + x (1 - d x) twice in double, which squares the error each time (2^-44, then the
// double rounding level).  Four FP64 instructions instead of an IEEE double division; the result
// may differ from the correctly rounded quotient in the last bit.
__device__ __forceinline__ double recip_nr(double d) {
  double x = widen_bits(__fdividef(1.0f, narrow_bits(d)));
  x = fma(x, fma(-d, x, 1.0), x);
  x = fma(x, fma(-d, x, 1.0), x);
  return x;
}

template <typename T> __device__ __forceinline__ double widen(T v);
template <> __device__ __forceinline__ double widen<float>(float v) { return f2d(v); }
template <> __device__ __forceinline__ double widen<double>(double v) { return v; }
template <typename T> __device__ __forceinline__ T narrow(double v);
template <> __device__ __forceinline__ float narrow<float>(double v) { return d2f(v); }
template <> __device__ __forceinline__ double narrow<double>(double v) { return v; }

// loads and stores of data touched once (evict-first in L1 and L2)
__device__ __forceinline__ cplx<float> ld_stream(const cplx<float>* p) {
  const float2 v = __ldcs(reinterpret_cast<const float2*>(p));
  return mk<float>(v.x, v.y);
}
__device__ __forceinline__ cplx<double> ld_stream(const cplx<double>* p) {
  const double2 v = __ldcs(reinterpret_cast<const double2*>(p));
  return mk<double>(v.x, v.y);
}
__device__ __forceinline__ void st_stream(cplx<float>* p, cplx<float> v) {
  __stcs(reinterpret_cast<float2*>(p), make_float2(v.x, v.y));
}
__device__ __forceinline__ void st_stream(cplx<double>* p, cplx<double> v) {
  __stcs(reinterpret_cast<double2*>(p), make_double2(v.x, v.y));
}

template <typename T> __device__ __forceinline__ cplx<double> wid(cplx<T> a) { return mk<double>(widen<T>(a.x), widen<T>(a.y)); }
template <typename T> __device__ __forceinline__ cplx<T> nar(cplx<double> a) { return mk<T>(narrow<T>(a.x), narrow<T>(a.y)); }

__device__ __forceinline__ cplx<double> cdiv(cplx<double> a, cplx<double> b) {
  const double den = b.x * b.x + b.y * b.y;
  return mk<double>((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

struct KInfo {
  int kxi, kyi;
  bool nyq, zero;
  double kx, ky, kk;
};

// thread i of a chunk (columns [kx0, kx0 + w), every ky) -> wavenumber column; kidx = kyi*nkx + kxi
__device__ __forceinline__ int64_t chunk_kidx(const Geometry& g, int64_t i, int kx0, int w) {
  const unsigned ii = (unsigned)i;  // total wavenumbers < 2^31
  const int kyi = (int)(ii / (unsigned)w);
  return (int64_t)kyi * g.nkx + kx0 + (int)(ii - (unsigned)kyi * (unsigned)w);
}

// per-block wavenumber table of the tiled kernels: grid column offset, kbuf index, k/2 components
struct KTile {
  int col[64];
  int kid[64];
  double hkx[64], hky[64];
  double kk[64];
};

__device__ __forceinline__ void fill_ktile(const Geometry& g, KTile& t, int64_t i0, int64_t total, int kx0, int w,
                                           int tk) {
  for (int kk = threadIdx.x; kk < tk; kk += blockDim.x) {
    const int64_t it = i0 + kk;
    int col = -1, kid = 0;
    double hx = 0.0, hy = 0.0;
    if (it < total) {
      const int64_t kidx = chunk_kidx(g, it, kx0, w);
      const unsigned ku = (unsigned)kidx;
      const int kyi = (int)(ku / (unsigned)g.nkx), kxi = (int)(ku - (unsigned)kyi * (unsigned)g.nkx);
      const bool nyq = ((g.nx % 2 == 0) && kxi == g.nx / 2) || ((g.ny % 2 == 0) && kyi == g.ny / 2);
      const int nyv = (kyi < (g.ny + 1) / 2) ? kyi : kyi - g.ny;
      col = kyi * g.pitch + kxi;
      kid = (int)kidx;
      hx = M_PI * (double)kxi / g.Lx;
      hy = M_PI * (double)nyv / g.Ly;
      if (nyq) kid = -1 - kid;  // flag Nyquist columns (negative), index recoverable
    }
    t.col[kk] = col;
    t.kid[kk] = kid;
    t.hkx[kk] = hx;
    t.hky[kk] = hy;
    t.kk[kk] = 2.0 * sqrt(hx * hx + hy * hy);
  }
}

__device__ __forceinline__ KInfo kinfo(const Geometry& g, int64_t kidx) {
  KInfo r;
  r.kxi = (int)(kidx % g.nkx);
  r.kyi = (int)(kidx / g.nkx);
  r.nyq = ((g.nx % 2 == 0) && r.kxi == g.nx / 2) || ((g.ny % 2 == 0) && r.kyi == g.ny / 2);
  r.zero = (r.kxi == 0 && r.kyi == 0);
  const int nyv = (r.kyi < (g.ny + 1) / 2) ? r.kyi : r.kyi - g.ny;
  r.kx = 2.0 * M_PI * (double)r.kxi / g.Lx;
  r.ky = 2.0 * M_PI * (double)nyv / g.Ly;
  r.kk = sqrt(r.kx * r.kx + r.ky * r.ky);
  return r;
}

// kinfo with the host's 2 pi / Lx and 2 pi / Ly, and 1 / |k| from one reciprocal square root (|k|
// as its product with |k|^2): no division on the FP64 pipe, which bounds the table solve
__device__ __forceinline__ KInfo kinfo_fast(const Geometry& g, int64_t kidx, double tpx, double tpy, double& ik) {
  KInfo r;
  const unsigned ku = (unsigned)kidx;  // wavenumbers < 2^31
  r.kyi = (int)(ku / (unsigned)g.nkx);
  r.kxi = (int)(ku - (unsigned)r.kyi * (unsigned)g.nkx);
  r.nyq = ((g.nx % 2 == 0) && r.kxi == g.nx / 2) || ((g.ny % 2 == 0) && r.kyi == g.ny / 2);
  r.zero = (r.kxi == 0 && r.kyi == 0);
  const int nyv = (r.kyi < (g.ny + 1) / 2) ? r.kyi : r.kyi - g.ny;
  r.kx = tpx * (double)r.kxi;
  r.ky = tpy * (double)nyv;
  const double k2 = r.kx * r.kx + r.ky * r.ky;
  ik = r.zero ? 0.0 : rsqrt(k2);
  r.kk = k2 * ik;
  return r;
}

// grid element (field f, plane c) of wavenumber column (kyi, kxi)
__device__ __forceinline__ size_t gidx(const Geometry& g, int f, int c, int kyi, int kxi) {
  return (((size_t)f * g.nz + c) * g.ny + kyi) * g.pitch + kxi;
}

// four consecutive table values (16-byte aligned)
__device__ __forceinline__ void ld4(const float* p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&o)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], c = reinterpret_cast<const double2*>(p)[1];
  o[0] = a.x; o[1] = a.y; o[2] = c.x; o[3] = c.y;
}

// stage a table into shared memory when it fits, else read it from global memory
template <typename T>
__device__ __forceinline__ const T* stage_table(T* sm, const T* gsrc, int count, bool use) {
  if (!use) return gsrc;
  for (int i = threadIdx.x; i < count; i += blockDim.x) sm[i] = gsrc[i];
  return sm;
}

// ---------------------------------------------------------------------------------------------
// forward: kbuf[o][n][k] = sum_c C[n][c] a_c + DC[n][c] b_c
// ---------------------------------------------------------------------------------------------
template <typename T, int NB>
__global__ void __launch_bounds__(kBvpThreads) fwd_kernel(Geometry g, const T* __restrict__ ct_g,
                                                          const T* __restrict__ dct_g, int npad, int smem_tabs,
                                                          const cplx<T>* __restrict__ grid, cplx<T>* __restrict__ kbuf,
                                                          const int* __restrict__ zrange, int kx0, int w) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = g.nz;
  T* sm = reinterpret_cast<T*>(smraw);
  const T* Ct = stage_table<T>(sm, ct_g, N * npad, smem_tabs != 0);
  const T* DCt = stage_table<T>(sm + N * npad, dct_g, N * npad, smem_tabs != 0);
  __syncthreads();
  const int64_t K = (int64_t)g.nkx * g.ny;
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= (int64_t)w * g.ny) return;
  const int64_t kidx = chunk_kidx(g, it, kx0, w);
  const KInfo ki = kinfo(g, kidx);
  if (ki.nyq) return;
  const int clo = zrange[0], chi = zrange[1];
  const T hkx = (T)(0.5 * ki.kx), hky = (T)(0.5 * ki.ky);
  const bool tq = g.spectral_curl != 0;
  for (int o = 0; o < 3; ++o) {
    const bool use_b = tq && o < 2;
    for (int n0 = 0; n0 < N; n0 += NB) {
      cplx<T> acc[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) acc[j] = mk<T>((T)0, (T)0);
      for (int c = clo; c <= chi; ++c) {
        cplx<T> a = grid[gidx(g, o, c, ki.kyi, ki.kxi)];
        cplx<T> b = mk<T>((T)0, (T)0);
        if (tq) {
          if (o == 0) {        // Fx + 1/2 i ky tz ;  - 1/2 D ty
            a = a + mul_i(scl(grid[gidx(g, 5, c, ki.kyi, ki.kxi)], hky));
            b = scl(grid[gidx(g, 4, c, ki.kyi, ki.kxi)], (T)-0.5);
          } else if (o == 1) { // Fy - 1/2 i kx tz ;  + 1/2 D tx
            a = a - mul_i(scl(grid[gidx(g, 5, c, ki.kyi, ki.kxi)], hkx));
            b = scl(grid[gidx(g, 3, c, ki.kyi, ki.kxi)], (T)0.5);
          } else {             // Fz + 1/2 (i kx ty - i ky tx)
            a = a + mul_i(scl(grid[gidx(g, 4, c, ki.kyi, ki.kxi)], hkx) -
                          scl(grid[gidx(g, 3, c, ki.kyi, ki.kxi)], hky));
          }
        }
        const T* crow = Ct + (size_t)c * npad + n0;
        const T* drow = DCt + (size_t)c * npad + n0;
#pragma unroll
        for (int j4 = 0; j4 < NB; j4 += 4) {
          T cm[4];
          ld4(crow + j4, cm);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            acc[j4 + q].x += cm[q] * a.x;
            acc[j4 + q].y += cm[q] * a.y;
          }
          if (use_b) {
            T dm[4];
            ld4(drow + j4, dm);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              acc[j4 + q].x += dm[q] * b.x;
              acc[j4 + q].y += dm[q] * b.y;
            }
          }
        }
      }
      const size_t base = ((size_t)o * N) * K + kidx;
#pragma unroll
      for (int j = 0; j < NB; ++j)
        if (n0 + j < N) kbuf[base + (size_t)(n0 + j) * K] = acc[j];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// FP64 solve
// ---------------------------------------------------------------------------------------------
struct SolveWs {
  cplx<double>* sw;   // [3][N][slots] sweep values
  double* fr;         // [3][N][slots] rho, t, folded boundary coefficient
  int slots;
};

// k = 0 (Sec. III.C, Eqs. 47-52; Appendix A, Eq. A12): w = 0; sigma c_n = -f_n/eta with the
// Dirichlet / Neumann (Robin with slip) rows on the truncated series; no pressure (not needed).
// The sweep values of the slot's workspace hold the scaled right-hand side meanwhile.
template <typename T, bool SLIP>
__device__ __noinline__ void zero_mode(const Geometry& g, const double* __restrict__ band, const T* __restrict__ bandT,
                                       cplx<T>* __restrict__ kbuf, cplx<T>* __restrict__ kaux,
                                       cplx<double>* __restrict__ sw, int slots, int slot, int64_t kidx, int64_t K) {
  const int N = g.nz;
  auto KB = [&](int f, int n) -> cplx<T>& { return kbuf[((size_t)f * N + n) * K + kidx]; };
  auto SW = [&](int f, int n) -> cplx<double>& { return sw[((size_t)f * N + n) * slots + slot]; };
  auto AUX = [&](int q) -> cplx<T>& { return kaux[(size_t)q * K + kidx]; };
  const double* bl = band;
  const double* bd = band + N;
  const double* bu = band + 2 * N;
  const double* bP = band + 3 * N;
  const double* bQ = band + 4 * N;
  (void)bandT;
  const double sH = 2.0 / g.H;
  const double sig = sH * sH;
  const double inv_eta = 1.0 / g.eta;
  for (int o = 0; o < 3; ++o) {
    if (g.mode == DPS_FREE || o == 2) {
      for (int n = 0; n < N; ++n) KB(o, n) = mk<T>((T)0, (T)0);
      continue;
    }
    cplx<double> Sp = mk<double>(0, 0), Sm = mk<double>(0, 0), Pd = mk<double>(0, 0), Pm = mk<double>(0, 0);
    for (int n = 0; n < N; ++n) {
      const cplx<double> cn = scl(wid(KB(o, n)), -inv_eta / sig);
      SW(0, n) = cn;
      const double sgn = (n & 1) ? -1.0 : 1.0;
      Sp = Sp + scl(cn, bQ[n]);
      Sm = Sm + scl(cn, sgn * bQ[n]);
      Pd = Pd + scl(cn, bP[n]);
      if (SLIP) Pm = Pm + scl(cn, sgn * bP[n]);
    }
    cplx<double> a0, a1;
    if (SLIP) {
      // Robin rows (Eq. A12): y(-1) - l0 (2/H) y_s(-1) = g_bot and, in the slit,
      // y(+1) + lH (2/H) y_s(+1) = g_top (above one wall: y_s(+1) = 0); y(+-1) = S+- + a0 +- a1,
      // y_s(+1) = Pd + a1, y_s(-1) = -Pm + a1; g = Nx Ny u^W (unnormalised transform)
      const double nxy = (double)g.nx * (double)g.ny;
      const double al = 1.0 + g.slip0 * sH;
      const cplx<double> Rb = mk<double>(nxy * g.uw0[o], 0.0) - Sm - scl(Pm, g.slip0 * sH);
      if (g.mode == DPS_BOTTOM_WALL) {
        a1 = scl(Pd, -1.0);
        a0 = Rb + scl(a1, al);
      } else {
        const double be = 1.0 + g.slipH * sH;
        const cplx<double> Rt = mk<double>(nxy * g.uwH[o], 0.0) - Sp - scl(Pd, g.slipH * sH);
        a1 = scl(Rt - Rb, 1.0 / (al + be));
        a0 = Rb + scl(a1, al);
      }
    } else if (g.mode == DPS_BOTTOM_WALL) {  // y(-1) = 0, y_s(+1) = 0
      a1 = scl(Pd, -1.0);
      a0 = a1 - Sm;
    } else {                           // y(-1) = y(+1) = 0
      a0 = scl(Sp + Sm, -0.5);
      a1 = scl(Sp - Sm, -0.5);
    }
    for (int n = 0; n < N; ++n) {
      cplx<double> y = scl(SW(0, n), bd[n]);
      if (n >= 2) y = y + scl(SW(0, n - 2), bl[n]);
      if (n + 2 < N) y = y + scl(SW(0, n + 2), bu[n]);
      if (n == 0) y = y + a0;
      if (n == 1) y = y + a1;
      KB(o, n) = nar<T>(y);
    }
  }
  for (int q = 0; q < 12; ++q) AUX(q) = mk<T>((T)0, (T)0);
}

// Wall-correction amplitudes (FP64 boundary rows) from the DP velocity at the walls (vtop, vbot)
// and, with slip, its z derivatives there: bottom wall Eqs. 41-44, slit Eqs. A4-A10 in closed
// form (reading B3), slip lengths and wall velocities Eqs. A3, A8.  Written to kaux as the
// node-value coefficients (cE + cG zeta) e^{-k zeta} + (tE + tG xi) e^{-k xi} per field.
template <typename T, bool SLIP>
__device__ __forceinline__ void wall_amplitudes(const Geometry& g, double kx, double ky, double kk, double ik,
                                                const cplx<double> (&vtop)[3], const cplx<double> (&vbot)[3],
                                                const cplx<double> (&dtop)[2], const cplx<double> (&dbot)[2],
                                                cplx<T>* __restrict__ kaux, int64_t kidx, int64_t K) {
  auto AUX = [&](int q) -> cplx<T>& { return kaux[(size_t)q * K + kidx]; };
  const double sH = g.sH;
  (void)dtop;
  (void)dbot;
  (void)sH;
  cplx<double> cE[3], cG[3], tE[3], tG[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) { cE[f] = cG[f] = tE[f] = tG[f] = mk<double>(0, 0); }
  if (g.mode != DPS_FREE) {
    const double ex = kx * ik, ey = ky * ik;  // ik = 1 / k
    auto Lp = [&](cplx<double> u, cplx<double> v) { return scl(u, ex) + scl(v, ey); };
    auto Tp = [&](cplx<double> u, cplx<double> v) { return scl(v, ex) - scl(u, ey); };
    // wall data (Eq. A3): minus the DP velocity, and with slip u_DP - l0 du_DP/dz at the bottom,
    // u_DP + lH du_DP/dz at the top for the tangential parts
    cplx<double> eb0 = vbot[0], eb1 = vbot[1], et0 = vtop[0], et1 = vtop[1];
    if (SLIP) {
      eb0 = eb0 - scl(dbot[0], g.slip0 * sH);
      eb1 = eb1 - scl(dbot[1], g.slip0 * sH);
      et0 = et0 + scl(dtop[0], g.slipH * sH);
      et1 = et1 + scl(dtop[1], g.slipH * sH);
    }
    const cplx<double> u0L = scl(Lp(eb0, eb1), -1.0), u0T = scl(Tp(eb0, eb1), -1.0);
    const cplx<double> w0 = scl(vbot[2], -1.0);
    cplx<double> AL = u0L, Az = w0, AT = u0T;
    cplx<double> BL = mk<double>(0, 0), Bz = mk<double>(0, 0), BT = mk<double>(0, 0);
    if (SLIP && g.mode == DPS_BOTTOM_WALL) {
      // bottom family only: Robin rows u - l0 du/dz = u0 with w(0) = w0 give
      // AT (1 + k l0) = u0T and AL (1 + 2 k l0) + i k l0 Az = u0L
      const double kl0 = kk * g.slip0;
      AT = scl(u0T, 1.0 / (1.0 + kl0));
      AL = scl(u0L - scl(mul_i(w0), kl0), 1.0 / (1.0 + 2.0 * kl0));
    }
    if (SLIP && g.mode == DPS_SLIT) {
      const cplx<double> uHL = scl(Lp(et0, et1), -1.0), uHT = scl(Tp(et0, et1), -1.0);
      const cplx<double> wH = scl(vtop[2], -1.0);
      const double kH = kk * g.H, E = exp(-kH), E2 = E * E;
      const double kl0 = kk * g.slip0, klH = kk * g.slipH;
      // transverse: [1 + k l0, E (1 - k l0); E (1 - k lH), 1 + k lH] [AT; BT] = [u0T; uHT]
      {
        const double t11 = 1.0 + kl0, t12 = E * (1.0 - kl0), t21 = E * (1.0 - klH), t22 = 1.0 + klH;
        const double idt = 1.0 / (t11 * t22 - t12 * t21);
        AT = scl(scl(u0T, t22) - scl(uHT, t12), idt);
        BT = scl(scl(uHT, t11) - scl(u0T, t21), idt);
      }
      // longitudinal/normal: S0 A + E N1 B = a0, SH B + E N2 A = b0 with A = (AL, Az), B = (BL, Bz),
      // S0 = [1 + 2 k l0, i k l0; 0, 1], SH = [1 + 2 k lH, -i k lH; 0, 1],
      // N1 = [(1 - k l0)(1 - kH) - k l0, i k (H (1 - k l0) + l0); i kH, 1 + kH],
      // N2 = [(1 - kH)(1 - k lH) - k lH, -i k (H (1 - k lH) + lH); -i kH, 1 + kH];
      // (S0 - E^2 N1 SH^-1 N2) A = a0 - E N1 SH^-1 b0, then B = SH^-1 (b0 - E N2 A)
      const cplx<double> zc = mk<double>(0, 0);
      const double sh = 1.0 / (1.0 + 2.0 * klH);
      const cplx<double> h11 = mk<double>(sh, 0), h12 = mk<double>(0, klH * sh);  // SH^-1 = [h11 h12; 0 1]
      const cplx<double> n11 = mk<double>((1.0 - kl0) * (1.0 - kH) - kl0, 0), n12 = mk<double>(0, kk * (g.H * (1.0 - kl0) + g.slip0));
      const cplx<double> n21 = mk<double>(0, kH), n22 = mk<double>(1.0 + kH, 0);
      const cplx<double> m11 = mk<double>((1.0 - kH) * (1.0 - klH) - klH, 0), m12 = mk<double>(0, -kk * (g.H * (1.0 - klH) + g.slipH));
      const cplx<double> m21 = mk<double>(0, -kH), m22 = mk<double>(1.0 + kH, 0);
      // P = SH^-1 N2, Q = N1 P
      const cplx<double> p11 = h11 * m11 + h12 * m21, p12 = h11 * m12 + h12 * m22, p21 = m21, p22 = m22;
      const cplx<double> q11 = n11 * p11 + n12 * p21, q12 = n11 * p12 + n12 * p22;
      const cplx<double> q21 = n21 * p11 + n22 * p21, q22 = n21 * p12 + n22 * p22;
      const cplx<double> x11 = mk<double>(1.0 + 2.0 * kl0, 0) - scl(q11, E2), x12 = mk<double>(0, kl0) - scl(q12, E2);
      const cplx<double> x21 = zc - scl(q21, E2), x22 = mk<double>(1.0, 0) - scl(q22, E2);
      const cplx<double> hb0 = h11 * uHL + h12 * wH, hb1 = wH;  // SH^-1 b0
      const cplx<double> r0 = u0L - scl(n11 * hb0 + n12 * hb1, E);
      const cplx<double> r1 = w0 - scl(n21 * hb0 + n22 * hb1, E);
      const cplx<double> det = x11 * x22 - x12 * x21;
      AL = cdiv(x22 * r0 - x12 * r1, det);
      Az = cdiv(x11 * r1 - x21 * r0, det);
      const cplx<double> e0 = uHL - scl(m11 * AL + m12 * Az, E), e1 = wH - scl(m21 * AL + m22 * Az, E);
      BL = h11 * e0 + h12 * e1;
      Bz = e1;
    }
    if (!SLIP && g.mode == DPS_SLIT) {
      const cplx<double> uHL = scl(Lp(vtop[0], vtop[1]), -1.0), uHT = scl(Tp(vtop[0], vtop[1]), -1.0);
      const cplx<double> wH = scl(vtop[2], -1.0);
      const double kH = kk * g.H;
      const double E = exp(-kH);
      const double E2 = E * E;
      // transverse: [1 E; E 1] [AT; BT] = [u0T; uHT]
      AT = scl(u0T - scl(uHT, E), 1.0 / (1.0 - E2));
      BT = scl(uHT - scl(u0T, E), 1.0 / (1.0 - E2));
      // longitudinal/normal: A = a0 - E M1 B, B = b0 - E M2 A  =>  (I - E^2 M1 M2) A = a0 - E M1 b0,
      // M1 = [[1-kH, i kH], [i kH, 1+kH]], M2 = [[1-kH, -i kH], [-i kH, 1+kH]]
      const double k2H2 = kH * kH;
      const cplx<double> m11 = mk<double>(1.0 - E2 * (1.0 - 2.0 * kH + 2.0 * k2H2), 0.0);
      const cplx<double> m12 = mk<double>(0.0, -E2 * 2.0 * k2H2);
      const cplx<double> m21 = mk<double>(0.0, E2 * 2.0 * k2H2);
      const cplx<double> m22 = mk<double>(1.0 - E2 * (1.0 + 2.0 * kH + 2.0 * k2H2), 0.0);
      const cplx<double> M1b_L = scl(uHL, 1.0 - kH) + scl(mul_i(wH), kH);
      const cplx<double> M1b_z = scl(mul_i(uHL), kH) + scl(wH, 1.0 + kH);
      const cplx<double> rL = u0L - scl(M1b_L, E);
      const cplx<double> rz = w0 - scl(M1b_z, E);
      const cplx<double> det = m11 * m22 - m12 * m21;
      AL = cdiv(m22 * rL - m12 * rz, det);
      Az = cdiv(m11 * rz - m21 * rL, det);
      const cplx<double> M2a_L = scl(AL, 1.0 - kH) - scl(mul_i(Az), kH);
      const cplx<double> M2a_z = scl(mul_i(AL), -kH) + scl(Az, 1.0 + kH);
      BL = uHL - scl(M2a_L, E);
      Bz = wH - scl(M2a_z, E);
    }
    // pressure amplitudes over 2 eta: bottom k (Az - i AL), top -k (Bz + i BL)
    const cplx<double> pib = scl(Az - mul_i(AL), kk);
    const cplx<double> pit = scl(Bz + mul_i(BL), -kk);
    // u_L = (AL - i pib zeta) e^{-k zeta} + (BL - i pit xi) e^{-k xi};  u_T = AT e^{-k zeta} + BT e^{-k xi}
    // w   = (Az + pib zeta) e^{-k zeta} + (Bz - pit xi) e^{-k xi}
    const cplx<double> gbL = scl(mul_i(pib), -1.0), gtL = scl(mul_i(pit), -1.0);
    cE[0] = scl(AL, ex) - scl(AT, ey);  cG[0] = scl(gbL, ex);
    tE[0] = scl(BL, ex) - scl(BT, ey);  tG[0] = scl(gtL, ex);
    cE[1] = scl(AL, ey) + scl(AT, ex);  cG[1] = scl(gbL, ey);
    tE[1] = scl(BL, ey) + scl(BT, ex);  tG[1] = scl(gtL, ey);
    cE[2] = Az;                          cG[2] = pib;
    tE[2] = Bz;                          tG[2] = scl(pit, -1.0);
  }
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    AUX(4 * f + 0) = nar<T>(cE[f]);
    AUX(4 * f + 1) = nar<T>(cG[f]);
    AUX(4 * f + 2) = nar<T>(tE[f]);
    AUX(4 * f + 3) = nar<T>(tG[f]);
  }
}

// FACT: factorise the banded systems while sweeping the pressure right-hand side and keep the
// factorisation in the slot's workspace; without FACT, reuse the factorisation left there by the
// previous call on the same slot, which must have had the same |k| (the partner -ky of a pair).
// Returns whether the slot now holds a factorisation.
template <typename T, bool FACT, bool SLIP>
__device__ __noinline__ bool solve_one(const Geometry& g, const double* __restrict__ band, const T* __restrict__ bandT,
                          cplx<T>* __restrict__ kbuf, cplx<T>* __restrict__ kaux, cplx<T>* __restrict__ pws,
                          cplx<double>* __restrict__ sw, double* __restrict__ fr, int slots, int slot, int64_t kidx,
                          int64_t K) {
  const int N = g.nz;
  const KInfo ki = kinfo(g, kidx);
  if (ki.nyq) return false;
  auto KB = [&](int f, int n) -> cplx<T>& { return kbuf[((size_t)f * N + n) * K + kidx]; };
  auto SW = [&](int f, int n) -> cplx<double>& { return sw[((size_t)f * N + n) * slots + slot]; };
  auto FR = [&](int f, int n) -> double& { return fr[((size_t)f * N + n) * slots + slot]; };
  auto PW = [&](int n) -> cplx<T>& { return pws[(size_t)n * slots + slot]; };
  auto AUX = [&](int q) -> cplx<T>& { return kaux[(size_t)q * K + kidx]; };
  const double* bl = band;
  const double* bd = band + N;
  const double* bu = band + 2 * N;
  const double* bP = band + 3 * N;
  const double* bQ = band + 4 * N;
  const T* tl = bandT;
  const T* td = bandT + N;
  const T* tu = bandT + 2 * N;
  const double sH = 2.0 / g.H;
  const double sig = sH * sH;
  const double inv_eta = 1.0 / g.eta;

  if (ki.zero) {
    zero_mode<T, SLIP>(g, band, bandT, kbuf, kaux, sw, slots, slot, kidx, K);
    return false;
  }

  const double kx = ki.kx, ky = ki.ky, kk = ki.kk, kap = kk * kk;
  const T tkx = (T)kx, tky = (T)ky, tsH = (T)sH, tie = (T)inv_eta;

  // Every sweep below loads the inputs of its next row before the FP64 recurrence of the current
  // row, so the memory latency of the workspace overlaps the dependent DFMA chain.
  const cplx<T> zT = mk<T>((T)0, (T)0);
  // ---- pressure: (D^2 - k^2) p = i kx f + i ky g + D h, DtN rows with zero data ----------------
  cplx<double> ptop = mk<double>(0, 0), pbot = mk<double>(0, 0);
  for (int par = 0; par < 2; ++par) {
    const int nlast = ((N - 1 - par) & 1) ? N - 2 : N - 1;
    cplx<double> s_next = mk<double>(0, 0), gacc = mk<double>(0, 0);
    double t_next = 0.0, bfold = 0.0;
    cplx<T> dh_next = zT;  // derivative recurrence of h over the opposite parity
    cplx<T> fc = KB(0, nlast), gc = KB(1, nlast), hc = (nlast + 1 < N) ? KB(2, nlast + 1) : zT;
    double rhoc = FACT ? 0.0 : FR(0, nlast), bcc = FACT ? 0.0 : FR(2, nlast);  // stored factorisation
    for (int n = nlast; n >= par; n -= 2) {
      cplx<T> fn = zT, gn = zT, hn = zT;
      double rhon = 0.0, bcn = 0.0;
      if (n - 2 >= par) {
        fn = KB(0, n - 2);
        gn = KB(1, n - 2);
        hn = KB(2, n - 1);
        if (!FACT) {
          rhon = FR(0, n - 2);
          bcn = FR(2, n - 2);
        }
      }
      cplx<T> dh = dh_next + scl(hc, (T)(2 * (n + 1)));
      dh_next = dh;
      if (n == 0) dh = scl(dh, (T)0.5);
      const cplx<T> rt = mk<T>(-tkx * fc.y - tky * gc.y + tsH * dh.x, tkx * fc.x + tky * gc.x + tsH * dh.y);
      const cplx<double> r = wid(rt);
      const double U = -kap * bu[n];
      const double bcur = FACT ? ((n == nlast) ? (sH * bP[n] + kk * bQ[n]) : bfold) : bcc;
      if (n > par) {
        double rho;
        if (FACT) {
          rho = recip_nr((sig - kap * bd[n]) - U * t_next);
          const double t = rho * (-kap * bl[n]);
          FR(0, n) = rho;
          FR(1, n) = t;
          FR(2, n) = bcur;
          bfold = (sH * bP[n - 2] + kk * bQ[n - 2]) - bcur * t;
          t_next = t;
        } else {
          rho = rhoc;
        }
        const cplx<double> s = scl(r - scl(s_next, U), rho);
        SW(0, n) = s;
        gacc = gacc - scl(s, bcur);
        s_next = s;
      } else {
        // row `par`: D' c - kappa a = r - U s_{par+2};  boundary row: beta_a a + bcur c = g'
        const double Dp = FACT ? (sig - kap * bd[n]) - U * t_next : rhoc;
        const double beta_a = (par == 0) ? kk : (sH + kk);
        const cplx<double> rhs = r - scl(s_next, U);
        const double idet = 1.0 / (Dp * beta_a + kap * bcur);
        const cplx<double> c0 = scl(scl(rhs, beta_a) + scl(gacc, kap), idet);
        const cplx<double> a = scl(scl(gacc, Dp) - scl(rhs, bcur), idet);
        if (FACT) {
          FR(0, n) = Dp;
          FR(2, n) = bcur;
        }
        // ascending substitution; y = B B c + a in the transform precision
        cplx<double> cm = c0;
        cplx<T> tcm2 = zT, tcm = nar<T>(c0);
        cplx<double> sp = scl(c0, bQ[par]);
        const cplx<T> ta = nar<T>(a);
        cplx<double> sc = (par + 2 <= nlast) ? SW(0, par + 2) : mk<double>(0, 0);
        double tc = (par + 2 <= nlast) ? FR(1, par + 2) : 0.0;
        for (int m = par + 2; m <= nlast + 2; m += 2) {
          cplx<double> sn = mk<double>(0, 0);
          double tn = 0.0;
          if (m + 2 <= nlast) {
            sn = SW(0, m + 2);
            tn = FR(1, m + 2);
          }
          cplx<T> tnew = zT;
          if (m <= nlast) {
            const cplx<double> cnew = sc - scl(cm, tc);
            sp = sp + scl(cnew, bQ[m]);
            cm = cnew;
            tnew = nar<T>(cnew);
          }
          const int q = m - 2;
          cplx<T> y = scl(tcm, td[q]) + scl(tnew, tu[q]);
          if (q >= 2) y = y + scl(tcm2, tl[q]);
          if (q == par) y = y + ta;
          PW(q) = y;
          tcm2 = tcm;
          tcm = tnew;
          sc = sn;
          tc = tn;
        }
        const double sgn = par ? -1.0 : 1.0;
        ptop = ptop + sp + a;
        pbot = pbot + scl(sp + a, sgn);
      }
      fc = fn;
      gc = gn;
      hc = hn;
      rhoc = rhon;
      bcc = bcn;
    }
  }

  // ---- velocity: three right-hand sides sharing the factorisation -------------------------------
  const double ik = 1.0 / kk;  // the one division per wavenumber
  const cplx<double> ik_top = scl(ptop, 0.5 * inv_eta * ik);
  const cplx<double> ik_bot = scl(pbot, 0.5 * inv_eta * ik);
  cplx<double> gt[3], gb[3];
  gt[0] = scl(mul_i(ik_top), -kx);
  gb[0] = scl(mul_i(ik_bot), kx);
  gt[1] = scl(mul_i(ik_top), -ky);
  gb[1] = scl(mul_i(ik_bot), ky);
  gt[2] = scl(ptop, 0.5 * inv_eta);
  gb[2] = scl(pbot, 0.5 * inv_eta);
  cplx<double> vtop[3], vbot[3];
  cplx<double> dtop[2], dbot[2];  // SLIP: y_s(+-1) of the tangential DP velocities
#pragma unroll
  for (int f = 0; f < 3; ++f) { vtop[f] = mk<double>(0, 0); vbot[f] = mk<double>(0, 0); }
#pragma unroll
  for (int f = 0; f < 2; ++f) { dtop[f] = mk<double>(0, 0); dbot[f] = mk<double>(0, 0); }
  for (int par = 0; par < 2; ++par) {
    const int nlast = ((N - 1 - par) & 1) ? N - 2 : N - 1;
    cplx<double> s_next[3], gacc[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      s_next[f] = mk<double>(0, 0);
      gacc[f] = par ? scl(gt[f] + gb[f], 0.5) : scl(gt[f] - gb[f], 0.5);
    }
    cplx<T> dp_next = zT;
    // current-row inputs, loaded one row ahead
    cplx<T> pc1 = (nlast + 1 < N) ? PW(nlast + 1) : zT, pc0 = PW(nlast);
    cplx<T> f0c = KB(0, nlast), f1c = KB(1, nlast), f2c = KB(2, nlast);
    double rhoc = FR(0, nlast), bc = FR(2, nlast);
    for (int n = nlast; n >= par; n -= 2) {
      cplx<T> pn1 = zT, pn0 = zT, f0n = zT, f1n = zT, f2n = zT;
      double rhon = 0.0, bn = 0.0;
      if (n - 2 >= par) {
        pn1 = PW(n - 1);
        pn0 = PW(n - 2);
        f0n = KB(0, n - 2);
        f1n = KB(1, n - 2);
        f2n = KB(2, n - 2);
        rhon = FR(0, n - 2);
        bn = FR(2, n - 2);
      }
      cplx<T> dp = dp_next + scl(pc1, (T)(2 * (n + 1)));
      dp_next = dp;
      if (n == 0) dp = scl(dp, (T)0.5);
      cplx<double> r[3];
      r[0] = wid(scl(scl(mul_i(pc0), tkx) - f0c, tie));
      r[1] = wid(scl(scl(mul_i(pc0), tky) - f1c, tie));
      r[2] = wid(scl(scl(dp, tsH) - f2c, tie));
      const double U = -kap * bu[n];
      const double bcur = bc;
      if (n > par) {
        const double rho = rhoc;
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          const cplx<double> s = scl(r[f] - scl(s_next[f], U), rho);
          SW(f, n) = s;
          gacc[f] = gacc[f] - scl(s, bcur);
          s_next[f] = s;
        }
      } else {
        const double Dp = rhoc;
        const double beta_a = (par == 0) ? kk : (sH + kk);
        const double idet = 1.0 / (Dp * beta_a + kap * bcur);
        const double sgn = par ? -1.0 : 1.0;
        cplx<double> cm[3];
        cplx<T> tcm2[3], tcm[3];
        cplx<double> sp[3], sd[2];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          const cplx<double> rhs = r[f] - scl(s_next[f], U);
          const cplx<double> c0 = scl(scl(rhs, beta_a) + scl(gacc[f], kap), idet);
          const cplx<double> a = scl(scl(gacc[f], Dp) - scl(rhs, bcur), idet);
          cm[f] = c0;
          tcm[f] = nar<T>(c0);
          tcm2[f] = zT;
          sp[f] = scl(c0, bQ[par]);
          if (SLIP && f < 2) {
            sd[f] = scl(c0, bP[par]);
            if (par) {  // a1 T_1 has y_s = a1 at both ends; a0 T_0 has none
              dtop[f] = dtop[f] + a;
              dbot[f] = dbot[f] + a;
            }
          }
          vtop[f] = vtop[f] + a;
          vbot[f] = vbot[f] + scl(a, sgn);
          gacc[f] = a;  // reuse: a_par of this field
        }
        // ascending substitution for the three fields together
        cplx<double> sc[3];
        double tc = (par + 2 <= nlast) ? FR(1, par + 2) : 0.0;
#pragma unroll
        for (int f = 0; f < 3; ++f) sc[f] = (par + 2 <= nlast) ? SW(f, par + 2) : mk<double>(0, 0);
        for (int m = par + 2; m <= nlast + 2; m += 2) {
          cplx<double> sn[3];
          double tn = 0.0;
#pragma unroll
          for (int f = 0; f < 3; ++f) sn[f] = mk<double>(0, 0);
          if (m + 2 <= nlast) {
#pragma unroll
            for (int f = 0; f < 3; ++f) sn[f] = SW(f, m + 2);
            tn = FR(1, m + 2);
          }
          const int q = m - 2;
#pragma unroll
          for (int f = 0; f < 3; ++f) {
            cplx<T> tnew = zT;
            if (m <= nlast) {
              const cplx<double> cnew = sc[f] - scl(cm[f], tc);
              sp[f] = sp[f] + scl(cnew, bQ[m]);
              if (SLIP && f < 2) sd[f] = sd[f] + scl(cnew, bP[m]);
              cm[f] = cnew;
              tnew = nar<T>(cnew);
            }
            cplx<T> y = scl(tcm[f], td[q]) + scl(tnew, tu[q]);
            if (q >= 2) y = y + scl(tcm2[f], tl[q]);
            if (q == par) y = y + nar<T>(gacc[f]);
            KB(f, q) = y;
            tcm2[f] = tcm[f];
            tcm[f] = tnew;
            sc[f] = sn[f];
          }
          tc = tn;
        }
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          vtop[f] = vtop[f] + sp[f];
          vbot[f] = vbot[f] + scl(sp[f], sgn);
        }
        if (SLIP) {  // T_n'(-1) = (-1)^(n+1) n^2: the even part enters y_s(-1) negated
#pragma unroll
          for (int f = 0; f < 2; ++f) {
            dtop[f] = dtop[f] + sd[f];
            dbot[f] = dbot[f] + scl(sd[f], -sgn);
          }
        }
      }
      pc1 = pn1;
      pc0 = pn0;
      f0c = f0n;
      f1c = f1n;
      f2c = f2n;
      rhoc = rhon;
      bc = bn;
    }
  }

  wall_amplitudes<T, SLIP>(g, kx, ky, kk, ik, vtop, vbot, dtop, dbot, kaux, kidx, K);
  return true;
}

template <typename T, bool SLIP>
__global__ void __launch_bounds__(kBvpThreads, 3) solve_kernel(Geometry g, const double* __restrict__ band,
                                                            const T* __restrict__ bandT, cplx<T>* __restrict__ kbuf,
                                                            cplx<T>* __restrict__ kaux, cplx<T>* __restrict__ pws,
                                                            cplx<double>* __restrict__ sw, double* __restrict__ fr,
                                                            int kx0, int w) {
  const int64_t K = (int64_t)g.nkx * g.ny;
  const int rows = g.ny / 2 + 1;  // ky rows 0 .. ny/2; row j > 0 pairs with ny - j unless 2 j = ny
  const int64_t total = (int64_t)w * rows;
  const int slots = gridDim.x * blockDim.x;
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t i = slot; i < total; i += slots) {
    const unsigned ii = (unsigned)i;
    const int kyi = (int)(ii / (unsigned)w);
    const int kxi = kx0 + (int)(ii - (unsigned)kyi * (unsigned)w);
    const int64_t k1 = (int64_t)kyi * g.nkx + kxi;
    const bool factored = solve_one<T, true, SLIP>(g, band, bandT, kbuf, kaux, pws, sw, fr, slots, slot, k1, K);
    if (kyi > 0 && 2 * kyi != g.ny && factored) {
      // the partner -ky has the same |k| and therefore the same banded systems
      const int64_t k2 = (int64_t)(g.ny - kyi) * g.nkx + kxi;
      solve_one<T, false, SLIP>(g, band, bandT, kbuf, kaux, pws, sw, fr, slots, slot, k2, K);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// FP64 solve from a plan-time factorisation table.  The banded systems of a wavenumber depend on
// |k| only, so their elimination coefficients are computed once per (kx, |ky|) when the plan is
// created (factor_kernel) and read by every product.  Each row's pivot reciprocal rho_n scales
// that row's right-hand side where the right-hand side is formed (in the transform precision, as
// the right-hand side itself), so the FP64 sweep of a row is s_n = r'_n - V_n s_{n+2},
// V_n = rho_n U_n: one DFMA per real right-hand side instead of a DFMA and a DMUL.
//
// Table fac[(n * 4 + q) * KP + kp], kp = |kyi| nkx + kxi, KP = nkx (ny/2 + 1); row n of parity
// par = n & 1:
//   n > par:  q0 V_n = U_n rho_n   q1 t_n   q2 b_n (folded boundary coefficient)   q3 rho_n
//   n = par:  q0 U_n               q1 D'    q2 b_n                                  q3 1/(D' beta_a + k^2 b_n)
// with U_n = -k^2 u_n, rho_n = 1/((sigma - k^2 d_n) - U_n t_{n+2}), t_n = -k^2 l_n rho_n, and the
// DtN boundary rows folded as in solve_one.
// ---------------------------------------------------------------------------------------------
__global__ void factor_kernel(Geometry g, const double* __restrict__ band, double* __restrict__ fac, int64_t KP) {
  const int64_t kp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (kp >= KP) return;
  const int N = g.nz;
  const int kxi = (int)(kp % g.nkx), kyi = (int)(kp / g.nkx);
  const double* bl = band;
  const double* bd = band + N;
  const double* bu = band + 2 * N;
  const double* bP = band + 3 * N;
  const double* bQ = band + 4 * N;
  const double kx = 2.0 * M_PI * (double)kxi / g.Lx, ky = 2.0 * M_PI * (double)kyi / g.Ly;
  const double kk = sqrt(kx * kx + ky * ky), kap = kk * kk;
  const double sH = 2.0 / g.H, sig = sH * sH;
  auto F = [&](int n, int q) -> double& { return fac[((size_t)n * 4 + q) * KP + kp]; };
  for (int par = 0; par < 2; ++par) {
    const int nlast = ((N - 1 - par) & 1) ? N - 2 : N - 1;
    double t_next = 0.0, bfold = 0.0;
    for (int n = nlast; n >= par; n -= 2) {
      const double U = -kap * bu[n];
      const double bcur = (n == nlast) ? (sH * bP[n] + kk * bQ[n]) : bfold;
      if (n > par) {
        const double rho = 1.0 / ((sig - kap * bd[n]) - U * t_next);
        const double t = rho * (-kap * bl[n]);
        F(n, 0) = U * rho;
        F(n, 1) = t;
        F(n, 2) = bcur;
        F(n, 3) = rho;
        bfold = (sH * bP[n - 2] + kk * bQ[n - 2]) - bcur * t;
        t_next = t;
      } else {
        const double Dp = (sig - kap * bd[n]) - U * t_next;
        const double beta_a = (par == 0) ? kk : (sH + kk);
        F(n, 0) = U;
        F(n, 1) = Dp;
        F(n, 2) = bcur;
        F(n, 3) = (kk > 0.0) ? 1.0 / (Dp * beta_a + kap * bcur) : 0.0;  // k = 0 takes zero_mode
      }
    }
  }
}

// r rho in the transform precision (the right-hand side's own precision), widened exactly
template <typename T> __device__ __forceinline__ cplx<double> prescale(cplx<T> r, double rho);
template <> __device__ __forceinline__ cplx<double> prescale<float>(cplx<float> r, double rho) {
  const float rf = narrow_bits(rho);
  return mk<double>(f2d(r.x * rf), f2d(r.y * rf));
}
template <> __device__ __forceinline__ cplx<double> prescale<double>(cplx<double> r, double rho) {
  return mk<double>(r.x * rho, r.y * rho);
}

template <typename T, bool SLIP>
__device__ __noinline__ void solve_tab(const Geometry& g, const double* __restrict__ band, const T* __restrict__ bandT,
                                       const double* __restrict__ fac, int64_t KP, cplx<T>* __restrict__ kbuf,
                                       cplx<T>* __restrict__ kaux, cplx<T>* __restrict__ pws,
                                       cplx<double>* __restrict__ sw, int slots, int slot, int64_t kidx, int64_t K,
                                       double tpx, double tpy) {
  const int N = g.nz;
  double ik;
  const KInfo ki = kinfo_fast(g, kidx, tpx, tpy, ik);
  if (ki.nyq) return;
  if (ki.zero) {
    zero_mode<T, SLIP>(g, band, bandT, kbuf, kaux, sw, slots, slot, kidx, K);
    return;
  }
  const int64_t kp = (int64_t)((2 * ki.kyi <= g.ny) ? ki.kyi : g.ny - ki.kyi) * g.nkx + ki.kxi;
  // the spectra are read once and written once: streaming loads and stores, so that they do not
  // push the sweep values out of L2
  auto KBL = [&](int f, int n) -> cplx<T> { return ld_stream(kbuf + ((size_t)f * N + n) * K + kidx); };
  auto KBS = [&](int f, int n, cplx<T> v) { st_stream(kbuf + ((size_t)f * N + n) * K + kidx, v); };
  // sweep values of one parity at a time: row n in slot n / 2, so a thread's live workspace is
  // half of the rows (kept small enough to stay in L2 across the sweep and the substitution)
  const int NH = (N + 1) / 2;
  auto SW = [&](int f, int n) -> cplx<double>& { return sw[((size_t)f * NH + (n >> 1)) * slots + slot]; };
  auto PW = [&](int n) -> cplx<T>& { return pws[(size_t)n * slots + slot]; };
  auto FAC = [&](int n, int q) -> double { return fac[((size_t)n * 4 + q) * KP + kp]; };
  const double* bP = band + 3 * N;
  const double* bQ = band + 4 * N;
  const T* tl = bandT;
  const T* td = bandT + N;
  const T* tu = bandT + 2 * N;
  const double sH = g.sH;
  const double inv_eta = g.inv_eta;
  const double kx = ki.kx, ky = ki.ky, kk = ki.kk, kap = kk * kk;
  const T tkx = (T)kx, tky = (T)ky, tsH = (T)sH, tie = (T)inv_eta;
  const cplx<T> zT = mk<T>((T)0, (T)0);

  // ---- pressure: (D^2 - k^2) p = i kx f + i ky g + D h, DtN rows with zero data ----------------
  cplx<double> ptop = mk<double>(0, 0), pbot = mk<double>(0, 0);
  for (int par = 0; par < 2; ++par) {
    const int nlast = ((N - 1 - par) & 1) ? N - 2 : N - 1;
    cplx<double> s_next = mk<double>(0, 0), gacc = mk<double>(0, 0);
    cplx<T> dh_next = zT;  // derivative recurrence of h over the opposite parity
    cplx<T> fc = KBL(0, nlast), gc = KBL(1, nlast), hc = (nlast + 1 < N) ? KBL(2, nlast + 1) : zT;
    double vc = FAC(nlast, 0), bc = FAC(nlast, 2), rc = FAC(nlast, 3);
    for (int n = nlast; n >= par; n -= 2) {
      cplx<T> fn = zT, gn = zT, hn = zT;
      double vn = 0.0, bn = 0.0, rn = 0.0;
      if (n - 2 >= par) {  // next row's inputs before this row's FP64 recurrence
        fn = KBL(0, n - 2);
        gn = KBL(1, n - 2);
        hn = KBL(2, n - 1);
        vn = FAC(n - 2, 0);
        bn = FAC(n - 2, 2);
        rn = FAC(n - 2, 3);
      }
      cplx<T> dh = dh_next + scl(hc, (T)(2 * (n + 1)));
      dh_next = dh;
      if (n == 0) dh = scl(dh, (T)0.5);
      const cplx<T> rt = mk<T>(-tkx * fc.y - tky * gc.y + tsH * dh.x, tkx * fc.x + tky * gc.x + tsH * dh.y);
      if (n > par) {
        const cplx<double> r = prescale<T>(rt, rc);
        const cplx<double> sv = mk<double>(fma(-vc, s_next.x, r.x), fma(-vc, s_next.y, r.y));
        SW(0, n) = sv;
        gacc = gacc - scl(sv, bc);
        s_next = sv;
      } else {
        // row `par`: D' c - kappa a = r - U s_{par+2};  boundary row: beta_a a + b c = g'
        const double U = vc, Dp = FAC(n, 1), idet = rc;
        const double beta_a = (par == 0) ? kk : (sH + kk);
        const cplx<double> rhs = wid(rt) - scl(s_next, U);
        // c0 = (beta_a rhs + kappa g) / det, a = (D' g - b rhs) / det, the 1/det folded into the
        // per-wavenumber constants
        const double cb = beta_a * idet, ck = kap * idet, cd = Dp * idet, cc = bc * idet;
        const cplx<double> c0 = scl(rhs, cb) + scl(gacc, ck);
        const cplx<double> a = scl(gacc, cd) - scl(rhs, cc);
        // ascending substitution; y = B B c + a in the transform precision
        cplx<double> cm = c0;
        cplx<T> tcm2 = zT, tcm = nar<T>(c0);
        cplx<double> sp = scl(c0, bQ[par]);
        const cplx<T> ta = nar<T>(a);
        cplx<double> sc = (par + 2 <= nlast) ? SW(0, par + 2) : mk<double>(0, 0);
        double tc = (par + 2 <= nlast) ? FAC(par + 2, 1) : 0.0;
        for (int m = par + 2; m <= nlast + 2; m += 2) {
          cplx<double> sn = mk<double>(0, 0);
          double tn = 0.0;
          if (m + 2 <= nlast) {
            sn = SW(0, m + 2);
            tn = FAC(m + 2, 1);
          }
          cplx<T> tnew = zT;
          if (m <= nlast) {
            const cplx<double> cnew = mk<double>(fma(-tc, cm.x, sc.x), fma(-tc, cm.y, sc.y));
            sp = sp + scl(cnew, bQ[m]);
            cm = cnew;
            tnew = nar<T>(cnew);
          }
          const int q = m - 2;
          cplx<T> y = scl(tcm, td[q]) + scl(tnew, tu[q]);
          if (q >= 2) y = y + scl(tcm2, tl[q]);
          if (q == par) y = y + ta;
          PW(q) = y;
          tcm2 = tcm;
          tcm = tnew;
          sc = sn;
          tc = tn;
        }
        ptop = ptop + sp + a;
        pbot = par ? pbot - (sp + a) : pbot + (sp + a);  // T_n(-1) = (-1)^n
      }
      fc = fn;
      gc = gn;
      hc = hn;
      vc = vn;
      bc = bn;
      rc = rn;
    }
  }

  // ---- velocity: three right-hand sides sharing the factorisation -------------------------------
  // the boundary data halved here (the parity split below takes half their sum or difference)
  const double qe = 0.25 * inv_eta, qk = qe * ik;
  const cplx<double> ik_top = scl(ptop, qk);
  const cplx<double> ik_bot = scl(pbot, qk);
  cplx<double> gt[3], gb[3];
  gt[0] = scl(mul_i(ik_top), -kx);
  gb[0] = scl(mul_i(ik_bot), kx);
  gt[1] = scl(mul_i(ik_top), -ky);
  gb[1] = scl(mul_i(ik_bot), ky);
  gt[2] = scl(ptop, qe);
  gb[2] = scl(pbot, qe);
  cplx<double> vtop[3], vbot[3];
  cplx<double> dtop[2], dbot[2];  // SLIP: y_s(+-1) of the tangential DP velocities
#pragma unroll
  for (int f = 0; f < 3; ++f) { vtop[f] = mk<double>(0, 0); vbot[f] = mk<double>(0, 0); }
#pragma unroll
  for (int f = 0; f < 2; ++f) { dtop[f] = mk<double>(0, 0); dbot[f] = mk<double>(0, 0); }
  for (int par = 0; par < 2; ++par) {
    const int nlast = ((N - 1 - par) & 1) ? N - 2 : N - 1;
    cplx<double> s_next[3], gacc[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      s_next[f] = mk<double>(0, 0);
      gacc[f] = par ? gt[f] + gb[f] : gt[f] - gb[f];
    }
    cplx<T> dp_next = zT;
    cplx<T> pc1 = (nlast + 1 < N) ? PW(nlast + 1) : zT, pc0 = PW(nlast);
    cplx<T> f0c = KBL(0, nlast), f1c = KBL(1, nlast), f2c = KBL(2, nlast);
    double vc = FAC(nlast, 0), bc = FAC(nlast, 2), rc = FAC(nlast, 3);
    for (int n = nlast; n >= par; n -= 2) {
      cplx<T> pn1 = zT, pn0 = zT, f0n = zT, f1n = zT, f2n = zT;
      double vn = 0.0, bn = 0.0, rn = 0.0;
      if (n - 2 >= par) {
        pn1 = PW(n - 1);
        pn0 = PW(n - 2);
        f0n = KBL(0, n - 2);
        f1n = KBL(1, n - 2);
        f2n = KBL(2, n - 2);
        vn = FAC(n - 2, 0);
        bn = FAC(n - 2, 2);
        rn = FAC(n - 2, 3);
      }
      cplx<T> dp = dp_next + scl(pc1, (T)(2 * (n + 1)));
      dp_next = dp;
      if (n == 0) dp = scl(dp, (T)0.5);
      cplx<T> rt[3];
      rt[0] = scl(scl(mul_i(pc0), tkx) - f0c, tie);
      rt[1] = scl(scl(mul_i(pc0), tky) - f1c, tie);
      rt[2] = scl(scl(dp, tsH) - f2c, tie);
      if (n > par) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          const cplx<double> r = prescale<T>(rt[f], rc);
          const cplx<double> sv = mk<double>(fma(-vc, s_next[f].x, r.x), fma(-vc, s_next[f].y, r.y));
          SW(f, n) = sv;
          gacc[f] = gacc[f] - scl(sv, bc);
          s_next[f] = sv;
        }
      } else {
        const double U = vc, Dp = FAC(n, 1), idet = rc;
        const double beta_a = (par == 0) ? kk : (sH + kk);
        const double cb = beta_a * idet, ck = kap * idet, cd = Dp * idet, cc = bc * idet;  // 1/det folded in
        cplx<double> cm[3];
        cplx<T> tcm2[3], tcm[3];
        cplx<double> sp[3], sd[2];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          const cplx<double> rhs = wid(rt[f]) - scl(s_next[f], U);
          const cplx<double> c0 = scl(rhs, cb) + scl(gacc[f], ck);
          const cplx<double> a = scl(gacc[f], cd) - scl(rhs, cc);
          cm[f] = c0;
          tcm[f] = nar<T>(c0);
          tcm2[f] = zT;
          sp[f] = scl(c0, bQ[par]);
          if (SLIP && f < 2) {
            sd[f] = scl(c0, bP[par]);
            if (par) {  // a1 T_1 has y_s = a1 at both ends; a0 T_0 has none
              dtop[f] = dtop[f] + a;
              dbot[f] = dbot[f] + a;
            }
          }
          vtop[f] = vtop[f] + a;
          vbot[f] = par ? vbot[f] - a : vbot[f] + a;  // T_n(-1) = (-1)^n
          gacc[f] = a;  // reuse: a_par of this field
        }
        // ascending substitution for the three fields together
        cplx<double> sc[3];
        double tc = (par + 2 <= nlast) ? FAC(par + 2, 1) : 0.0;
#pragma unroll
        for (int f = 0; f < 3; ++f) sc[f] = (par + 2 <= nlast) ? SW(f, par + 2) : mk<double>(0, 0);
        for (int m = par + 2; m <= nlast + 2; m += 2) {
          cplx<double> sn[3];
          double tn = 0.0;
#pragma unroll
          for (int f = 0; f < 3; ++f) sn[f] = mk<double>(0, 0);
          if (m + 2 <= nlast) {
#pragma unroll
            for (int f = 0; f < 3; ++f) sn[f] = SW(f, m + 2);
            tn = FAC(m + 2, 1);
          }
          const int q = m - 2;
#pragma unroll
          for (int f = 0; f < 3; ++f) {
            cplx<T> tnew = zT;
            if (m <= nlast) {
              const cplx<double> cnew = mk<double>(fma(-tc, cm[f].x, sc[f].x), fma(-tc, cm[f].y, sc[f].y));
              sp[f] = sp[f] + scl(cnew, bQ[m]);
              if (SLIP && f < 2) sd[f] = sd[f] + scl(cnew, bP[m]);
              cm[f] = cnew;
              tnew = nar<T>(cnew);
            }
            cplx<T> y = scl(tcm[f], td[q]) + scl(tnew, tu[q]);
            if (q >= 2) y = y + scl(tcm2[f], tl[q]);
            if (q == par) y = y + nar<T>(gacc[f]);
            KBS(f, q, y);
            tcm2[f] = tcm[f];
            tcm[f] = tnew;
            sc[f] = sn[f];
          }
          tc = tn;
        }
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          vtop[f] = vtop[f] + sp[f];
          vbot[f] = par ? vbot[f] - sp[f] : vbot[f] + sp[f];
        }
        if (SLIP) {  // T_n'(-1) = (-1)^(n+1) n^2: the even part enters y_s(-1) negated
#pragma unroll
          for (int f = 0; f < 2; ++f) {
            dtop[f] = dtop[f] + sd[f];
            dbot[f] = par ? dbot[f] + sd[f] : dbot[f] - sd[f];
          }
        }
      }
      pc1 = pn1;
      pc0 = pn0;
      f0c = f0n;
      f1c = f1n;
      f2c = f2n;
      vc = vn;
      bc = bn;
      rc = rn;
    }
  }
  wall_amplitudes<T, SLIP>(g, kx, ky, kk, ik, vtop, vbot, dtop, dbot, kaux, kidx, K);
}

// thread i of a chunk -> wavenumber, with the ky rows in the order 0, 1, ny-1, 2, ny-2, ...: the
// two wavenumbers (kx, +-ky) that read the same factorisation-table rows run in the same pass of the
// persistent grid, so the second read comes from L2
__device__ __forceinline__ int64_t paired_kidx(const Geometry& g, int64_t i, int kx0, int w) {
  const unsigned ii = (unsigned)i;
  const int j = (int)(ii / (unsigned)w);
  const int kyi = (j == 0) ? 0 : ((j & 1) ? (j + 1) >> 1 : g.ny - (j >> 1));
  return (int64_t)kyi * g.nkx + kx0 + (int)(ii - (unsigned)j * (unsigned)w);
}

// one thread per wavenumber of the chunk (persistent grid)
template <typename T, bool SLIP>
__global__ void __launch_bounds__(kBvpThreads, 3) solve_tab_kernel(Geometry g, const double* __restrict__ band,
                                                                const T* __restrict__ bandT,
                                                                const double* __restrict__ fac, int64_t KP,
                                                                cplx<T>* __restrict__ kbuf, cplx<T>* __restrict__ kaux,
                                                                cplx<T>* __restrict__ pws, cplx<double>* __restrict__ sw,
                                                                int kx0, int w, double tpx, double tpy) {
  const int64_t K = (int64_t)g.nkx * g.ny;
  const int64_t total = (int64_t)w * g.ny;
  const int slots = gridDim.x * blockDim.x;
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t i = slot; i < total; i += slots)
    solve_tab<T, SLIP>(g, band, bandT, fac, KP, kbuf, kaux, pws, sw, slots, slot, paired_kidx(g, i, kx0, w), K, tpx,
                       tpy);
}

// ---------------------------------------------------------------------------------------------
// backward: node values = IC y + correction(z_c); half-curl from ICD y + SD correction(nodes)
// ---------------------------------------------------------------------------------------------
template <typename T, int CB, bool CURL>
__global__ void __launch_bounds__(kBvpThreads) bwd_kernel(Geometry g, const T* __restrict__ ict_g,
                                                          const T* __restrict__ icdt_g, const T* __restrict__ sdt_g,
                                                          const T* __restrict__ zeta_g, int cpad, int smem_tabs,
                                                          const cplx<T>* __restrict__ kbuf,
                                                          const cplx<T>* __restrict__ kaux, cplx<T>* __restrict__ grid,
                                                          const int* __restrict__ zrange, int kx0, int w) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = g.nz;
  T* sm = reinterpret_cast<T*>(smraw);
  const int tab = N * cpad;
  const T* ICt = stage_table<T>(sm, ict_g, tab, smem_tabs != 0);
  const T* ICDt = CURL ? stage_table<T>(sm + tab, icdt_g, tab, smem_tabs != 0) : nullptr;
  const T* SDt = CURL ? stage_table<T>(sm + 2 * tab, sdt_g, tab, smem_tabs != 0) : nullptr;
  __syncthreads();
  const int64_t K = (int64_t)g.nkx * g.ny;
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= (int64_t)w * g.ny) return;
  const int64_t kidx = chunk_kidx(g, it, kx0, w);
  const KInfo ki = kinfo(g, kidx);
  const int clo = zrange[0], chi = zrange[1];
  const int nfo = CURL ? 6 : 3;
  if (ki.nyq) {
    for (int f = 0; f < nfo; ++f)
      for (int c = clo; c <= chi; ++c) grid[gidx(g, f, c, ki.kyi, ki.kxi)] = mk<T>((T)0, (T)0);
    return;
  }
  const T scale = (T)(1.0 / ((double)g.nx * (double)g.ny));
  const T kt = (T)ki.kk, H = (T)g.H;
  const bool corr = (g.mode != DPS_FREE) && !ki.zero;
  const bool top = (g.mode == DPS_SLIT);
  cplx<T> aE[3], aG[3], bE[3], bG[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    aE[f] = corr ? kaux[(size_t)(4 * f + 0) * K + kidx] : mk<T>((T)0, (T)0);
    aG[f] = corr ? kaux[(size_t)(4 * f + 1) * K + kidx] : mk<T>((T)0, (T)0);
    bE[f] = corr ? kaux[(size_t)(4 * f + 2) * K + kidx] : mk<T>((T)0, (T)0);
    bG[f] = corr ? kaux[(size_t)(4 * f + 3) * K + kidx] : mk<T>((T)0, (T)0);
  }
  // correction of field f at node j: (aE + aG zeta) e^{-k zeta} + (bE + bG xi) e^{-k xi}
  auto corr_at = [&](int f, T zt, T eb, T et) -> cplx<T> {
    cplx<T> v = scl(aE[f] + scl(aG[f], zt), eb);
    if (top) v = v + scl(bE[f] + scl(bG[f], H - zt), et);
    return v;
  };
  auto expk = [&](T z) -> T { return (sizeof(T) == 4) ? (T)expf((float)(-kt * z)) : (T)exp((double)(-kt * z)); };
  const T hkx = (T)(0.5 * ki.kx), hky = (T)(0.5 * ki.ky);
  for (int c0 = clo & ~3; c0 <= chi; c0 += CB) {  // 16-byte aligned table rows
    cplx<T> au[CB], av[CB], aw[CB], du[CB], dv[CB];
#pragma unroll
    for (int j = 0; j < CB; ++j) {
      au[j] = av[j] = aw[j] = mk<T>((T)0, (T)0);
      du[j] = dv[j] = mk<T>((T)0, (T)0);
    }
    for (int n = 0; n < N; ++n) {
      const cplx<T> yu = kbuf[((size_t)0 * N + n) * K + kidx];
      const cplx<T> yv = kbuf[((size_t)1 * N + n) * K + kidx];
      const cplx<T> yw = kbuf[((size_t)2 * N + n) * K + kidx];
      const T* irow = ICt + (size_t)n * cpad + c0;
      const T* drow = CURL ? ICDt + (size_t)n * cpad + c0 : nullptr;
#pragma unroll
      for (int j4 = 0; j4 < CB; j4 += 4) {
        T im[4];
        ld4(irow + j4, im);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = j4 + q;
          au[j].x += im[q] * yu.x; au[j].y += im[q] * yu.y;
          av[j].x += im[q] * yv.x; av[j].y += im[q] * yv.y;
          aw[j].x += im[q] * yw.x; aw[j].y += im[q] * yw.y;
        }
        if (CURL) {
          T dm[4];
          ld4(drow + j4, dm);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int j = j4 + q;
            du[j].x += dm[q] * yu.x; du[j].y += dm[q] * yu.y;
            dv[j].x += dm[q] * yv.x; dv[j].y += dm[q] * yv.y;
          }
        }
      }
    }
    if (corr && CURL) {
      // derivative of the interpolant of the correction node values (spectral differentiation)
      for (int jn = 0; jn < N; ++jn) {
        const T zt = zeta_g[jn];
        const T eb = expk(zt);
        const T et = top ? expk(H - zt) : (T)0;
        const cplx<T> cu = corr_at(0, zt, eb, et), cv = corr_at(1, zt, eb, et);
        const T* srow = SDt + (size_t)jn * cpad + c0;
#pragma unroll
        for (int j4 = 0; j4 < CB; j4 += 4) {
          T sd[4];
          ld4(srow + j4, sd);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int j = j4 + q;
            du[j].x += sd[q] * cu.x; du[j].y += sd[q] * cu.y;
            dv[j].x += sd[q] * cv.x; dv[j].y += sd[q] * cv.y;
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < CB; ++j) {
      const int c = c0 + j;
      if (c > chi) break;
      if (c < clo) continue;
      cplx<T> u = au[j], v = av[j], w = aw[j];
      if (corr) {
        const T zt = zeta_g[c];
        const T eb = expk(zt);
        const T et = top ? expk(H - zt) : (T)0;
        u = u + corr_at(0, zt, eb, et);
        v = v + corr_at(1, zt, eb, et);
        w = w + corr_at(2, zt, eb, et);
      }
      grid[gidx(g, 0, c, ki.kyi, ki.kxi)] = scl(u, scale);
      grid[gidx(g, 1, c, ki.kyi, ki.kxi)] = scl(v, scale);
      grid[gidx(g, 2, c, ki.kyi, ki.kxi)] = scl(w, scale);
      if (CURL) {
        // omega = 1/2 (i ky w - Dv, Du - i kx w, i kx v - i ky u)
        const cplx<T> ox = scl(mul_i(w), hky) - scl(dv[j], (T)0.5);
        const cplx<T> oy = scl(du[j], (T)0.5) - scl(mul_i(w), hkx);
        const cplx<T> oz = scl(mul_i(v), hkx) - scl(mul_i(u), hky);
        grid[gidx(g, 3, c, ki.kyi, ki.kxi)] = scl(ox, scale);
        grid[gidx(g, 4, c, ki.kyi, ki.kxi)] = scl(oy, scale);
        grid[gidx(g, 5, c, ki.kyi, ki.kxi)] = scl(oz, scale);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Lane-per-wavenumber forms of the two transforms (N <= 128).  A block owns 32 consecutive
// wavenumbers of the chunk, one per lane, and its warps split the output rows in groups of PG
// (Chebyshev index n forward, occupied plane backward).  The per-wavenumber operands sit in shared
// memory and are read one value per lane; the table rows sit beside them and are read as warp-wide
// broadcasts, so every shared load feeds PG or more FMAs and no table is read from global memory
// inside the contraction loops.
// ---------------------------------------------------------------------------------------------
constexpr int kLaneK = 32;
// Chebyshev rows per warp of the forward transform: 8 (float) while the block stays within the thread
// limit (nz <= 96), else 12; the smaller split needs fewer registers (74 against 142) and fits
// three blocks per SM
template <typename T> __host__ __device__ constexpr int fwd_pg() { return sizeof(T) == 4 ? 8 : 6; }
template <typename T> __host__ __device__ constexpr int fwd_pg_wide() { return sizeof(T) == 4 ? 12 : 6; }
template <typename T> __host__ __device__ constexpr int bwd_pg() { return sizeof(T) == 4 ? 8 : 4; }
template <typename T> __host__ __device__ constexpr int bwd_warps() { return sizeof(T) == 4 ? 5 : 10; }

// PG consecutive shared-memory table values (16-byte aligned) into registers
// (PG a multiple of 4 for float, of 2 for double)
template <int PG>
__device__ __forceinline__ void ld_row(const float* p, float (&o)[PG]) {
  static_assert(PG % 4 == 0, "float rows load as float4");
#pragma unroll
  for (int q = 0; q < PG; q += 4) {
    const float4 v = *reinterpret_cast<const float4*>(p + q);
    o[q] = v.x; o[q + 1] = v.y; o[q + 2] = v.z; o[q + 3] = v.w;
  }
}
template <int PG>
__device__ __forceinline__ void ld_row(const double* p, double (&o)[PG]) {
  static_assert(PG % 2 == 0, "double rows load as double2");
#pragma unroll
  for (int q = 0; q < PG; q += 2) {
    const double2 v = *reinterpret_cast<const double2*>(p + q);
    o[q] = v.x; o[q + 1] = v.y;
  }
}

// forward: kbuf[o][n][k] = sum_c C[n][c] a_o(c, k) + DC[n][c] b_o(c, k) over the occupied planes, with
// a_o = f_o + (1/2)(i k x tau)_o and the derivative terms of the half-curl b_x = -tau_y/2, b_y = tau_x/2.
// The planes stream through two shared-memory slots of cz planes (cp.async, double-buffered).
template <typename T> __host__ __device__ constexpr int fwd_max_threads() { return sizeof(T) == 4 ? 384 : 512; }

// MB = 3: the compact instantiation for blocks of at most 9 warps (nz <= 72 at 8 rows per warp) of
// the six-field form, compiled for three resident blocks per SM (registers are allocated 8 per thread at a time, so
// 76 would round up to 80 and leave room for two 9-warp blocks only).  MB = 0: the thread limit
// alone bounds the compilation.
constexpr int kFwdCompactThreads = 288;
template <typename T, int PG, bool TQ, int MB = 0>
__global__ void __launch_bounds__(MB == 3 ? kFwdCompactThreads : fwd_max_threads<T>(), MB) fwd_lane_kernel(Geometry g, const T* __restrict__ ct,
                                                                        const T* __restrict__ dct, int npad,
                                                                        const cplx<T>* __restrict__ grid,
                                                                        cplx<T>* __restrict__ kbuf,
                                                                        const int* __restrict__ zrange, int kx0, int w,
                                                                        int cz) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ KTile kt;
  constexpr int NF = TQ ? 6 : 3;  // staged fields per (plane, wavenumber); the first 3 (5) become a (a, b)
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int nthreads = blockDim.x;
  const int nwarps = nthreads >> 5;
  const int NP = nwarps * PG;  // rows covered by the block (>= N)
  const int N = g.nz;
  // two slots of cz planes each: field values [cz][NF][32] and table rows [cz][2][NP]
  const int slotV = cz * NF * kLaneK, slotM = cz * 2 * NP;
  cplx<T>* sVs = reinterpret_cast<cplx<T>*>(smraw);
  T* sMs = reinterpret_cast<T*>(sVs + 2 * (size_t)slotV);
  const int64_t K = (int64_t)g.nkx * g.ny;
  fill_ktile(g, kt, (int64_t)blockIdx.x * kLaneK, (int64_t)w * g.ny, kx0, w, kLaneK);
  __syncthreads();
  const int clo = zrange[0], chi = zrange[1];
  const size_t plane = (size_t)g.ny * g.pitch;
  const int col = kt.col[lane];
  const T hkx = (T)kt.hkx[lane], hky = (T)kt.hky[lane];  // k/2, narrowed once (not per plane)
  cplx<T> acc[3][PG];
#pragma unroll
  for (int o = 0; o < 3; ++o)
#pragma unroll
    for (int p = 0; p < PG; ++p) acc[o][p] = mk<T>((T)0, (T)0);
  const int nq = chi >= clo ? (chi - clo + cz) / cz : 0;  // plane chunks
  // copies of plane chunk q into slot q & 1 (warps stride over rows, lanes over wavenumbers)
  auto stage = [&](int q) {
    const int c0 = clo + q * cz, nc = min(cz, chi - c0 + 1);
    cplx<T>* sV = sVs + (q & 1) * (size_t)slotV;
    T* sM = sMs + (q & 1) * (size_t)slotM;
    for (int r = wi; r < nc * NF; r += nwarps) {
      const int cl = r / NF, f = r - cl * NF;  // NF is a compile-time constant
      cplx<T>* dst = sV + (size_t)r * kLaneK + lane;
      if (col >= 0) async_elem(dst, grid + ((size_t)f * g.nz + c0 + cl) * plane + col);
      else *dst = mk<T>((T)0, (T)0);
    }
    for (int cl = wi; cl < nc; cl += nwarps) {
      const T* crow = ct + (size_t)(c0 + cl) * npad;
      const T* drow = dct + (size_t)(c0 + cl) * npad;
      T* dst = sM + (size_t)cl * 2 * NP;
      for (int n = lane; n < NP; n += 32) {
        if (n < N) async_elem(dst + n, crow + n);
        else dst[n] = (T)0;
        if (TQ) {
          if (n < N) async_elem(dst + NP + n, drow + n);
          else dst[NP + n] = (T)0;
        }
      }
    }
    cp_commit();
  };
  if (nq > 0) stage(0);
  for (int q = 0; q < nq; ++q) {
    if (q + 1 < nq) {
      stage(q + 1);
      cp_wait_but_newest();
    } else {
      cp_wait_all();
    }
    __syncthreads();  // chunk q visible
    const int nc = min(cz, chi - (clo + q * cz) + 1);
    cplx<T>* sV = sVs + (q & 1) * (size_t)slotV;
    const T* sM = sMs + (q & 1) * (size_t)slotM;
    if (TQ) {
      // a_o = f_o + (1/2)(i k x tau)_o in slots 0..2, b_x = -tau_y/2, b_y = tau_x/2 in slots 3, 4
      for (int cl = wi; cl < nc; cl += nwarps) {
        cplx<T>* v = sV + (size_t)cl * NF * kLaneK + lane;
        const cplx<T> tx = v[3 * kLaneK], ty = v[4 * kLaneK], tz = v[5 * kLaneK];
        v[0] = v[0] + mul_i(scl(tz, hky));
        v[kLaneK] = v[kLaneK] - mul_i(scl(tz, hkx));
        v[2 * kLaneK] = v[2 * kLaneK] + mul_i(scl(ty, hkx) - scl(tx, hky));
        v[3 * kLaneK] = scl(ty, (T)-0.5);
        v[4 * kLaneK] = scl(tx, (T)0.5);
      }
      __syncthreads();
    }
    for (int cl = 0; cl < nc; ++cl) {
      const cplx<T>* vr = sV + (size_t)cl * NF * kLaneK + lane;
      const cplx<T> a0 = vr[0], a1 = vr[kLaneK], a2 = vr[2 * kLaneK];
      T cm[PG];
      ld_row<PG>(sM + (size_t)cl * 2 * NP + wi * PG, cm);
#pragma unroll
      for (int p = 0; p < PG; ++p) {
        acc[0][p].x += cm[p] * a0.x; acc[0][p].y += cm[p] * a0.y;
        acc[1][p].x += cm[p] * a1.x; acc[1][p].y += cm[p] * a1.y;
        acc[2][p].x += cm[p] * a2.x; acc[2][p].y += cm[p] * a2.y;
      }
      if (TQ) {
        const cplx<T> b0 = vr[3 * kLaneK], b1 = vr[4 * kLaneK];
        T dm[PG];
        ld_row<PG>(sM + (size_t)cl * 2 * NP + NP + wi * PG, dm);
#pragma unroll
        for (int p = 0; p < PG; ++p) {
          acc[0][p].x += dm[p] * b0.x; acc[0][p].y += dm[p] * b0.y;
          acc[1][p].x += dm[p] * b1.x; acc[1][p].y += dm[p] * b1.y;
        }
      }
    }
    __syncthreads();  // slot q & 1 may be refilled by the next iteration's copies
  }
  if (col >= 0) {
    const int kid = kt.kid[lane] >= 0 ? kt.kid[lane] : -1 - kt.kid[lane];
#pragma unroll
    for (int p = 0; p < PG; ++p) {
      const int n = wi * PG + p;
      if (n < N) {
#pragma unroll
        for (int o = 0; o < 3; ++o) kbuf[((size_t)o * N + n) * K + kid] = acc[o][p];
      }
    }
  }
}

// backward: node values on the occupied planes, u_f(z_c) = sum_n IC[c][n] y_f[n] + corr_f(z_c), with
// corr_f = (cE + cG zeta) e^{-k zeta} (+ (tE + tG xi) e^{-k xi} between two walls); with torques the
// half-curl (Eq. 11) from ICD y and the spectral derivative SD corr of the correction node values.
// CORR: 0 no wall, 1 bottom wall, 2 both walls.  The coefficients y and the table rows stream
// through shared memory in chunks of kBwdRows rows, double-buffered with cp.async, so the copies of
// chunk q + 1 overlap the contraction over chunk q.
constexpr int kBwdRows = 16;

template <typename T, int PG, bool CURL, int CORR>
__global__ void __launch_bounds__(32 * bwd_warps<T>(), sizeof(T) == 4 ? 3 : 1) bwd_lane_kernel(Geometry g, const T* __restrict__ ict,
                                                        const T* __restrict__ icdt, const T* __restrict__ sdt,
                                                        int cpad, const T* __restrict__ zeta_g,
                                                        const cplx<T>* __restrict__ kbuf,
                                                        const cplx<T>* __restrict__ kaux, cplx<T>* __restrict__ grid,
                                                        const int* __restrict__ zrange, int kx0, int w) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ KTile kt;
  constexpr bool DE = CURL && CORR > 0;              // derivative of the correction
  constexpr int NT = CURL ? (CORR > 0 ? 3 : 2) : 1;  // staged tables: IC, ICD, SD
  constexpr int NW = bwd_warps<T>();
  constexpr int CZ = NW * PG;  // planes per plane chunk (the block has NW warps)
  constexpr int RC = kBwdRows;
  constexpr int SLOT_Y = 3 * RC * kLaneK;  // complex values of y per slot  [3][RC][32]
  constexpr int SLOT_M = RC * NT * CZ;     // table values per slot        [RC][NT][CZ]
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int N = g.nz;
  const int N4 = (N + 3) & ~3;
  cplx<T>* sAmp = reinterpret_cast<cplx<T>*>(smraw);                                  // [12][32]
  cplx<T>* sYs = sAmp + (CORR ? 12 * kLaneK : 0);                                     // [2][SLOT_Y]
  T* sMs = reinterpret_cast<T*>(sYs + 2 * SLOT_Y);                                    // [2][SLOT_M]
  T* sE = sMs + 2 * SLOT_M;                                                            // [N][32] e^{-k zeta_j}
  T* sZ = sE + (CORR ? (size_t)N * kLaneK : 0);                                        // [N4] zeta_j
  const int64_t K = (int64_t)g.nkx * g.ny;
  fill_ktile(g, kt, (int64_t)blockIdx.x * kLaneK, (int64_t)w * g.ny, kx0, w, kLaneK);
  __syncthreads();
  const int col = kt.col[lane];
  const int kidl = kt.kid[lane];
  if (CORR) {
    for (int q = wi; q < 12; q += NW) {
      cplx<T>* dst = sAmp + q * kLaneK + lane;
      if (col >= 0 && kidl > 0) async_elem(dst, kaux + (size_t)q * K + kidl);
      else *dst = mk<T>((T)0, (T)0);
    }
    const T kk = (T)kt.kk[lane];
    for (int j = wi; j < N; j += NW) {
      const T kz = kk * zeta_g[j];
      sE[j * kLaneK + lane] = (col >= 0) ? ((sizeof(T) == 4) ? (T)expf((float)-kz) : (T)exp((double)-kz)) : (T)0;
    }
    for (int j = threadIdx.x; j < N4; j += blockDim.x) sZ[j] = j < N ? zeta_g[j] : (T)0;
  }
  cp_commit();  // the amplitudes form their own group
  const int clo = zrange[0], chi = zrange[1];
  const size_t plane = (size_t)g.ny * g.pitch;
  const size_t fstride = (size_t)g.nz * plane;
  const T scale = (T)(1.0 / ((double)g.nx * (double)g.ny));
  const T hkx = (T)kt.hkx[lane], hky = (T)kt.hky[lane];
  const int nq = (N + RC - 1) / RC;
  // copies of row chunk q (rows q RC .. q RC + RC - 1) for the plane chunk starting at c0
  auto stage = [&](int q, int c0) {
    cplx<T>* dY = sYs + (q & 1) * SLOT_Y;
    T* dM = sMs + (q & 1) * SLOT_M;
    const int n0 = q * RC;
    for (int r = wi; r < 3 * RC; r += NW) {
      const int f = r / RC, nn = r - f * RC;  // RC is a compile-time constant
      const int n = n0 + nn;
      cplx<T>* dst = dY + r * kLaneK + lane;
      if (n < N && col >= 0 && kidl >= 0) async_elem(dst, kbuf + ((size_t)f * N + n) * K + kidl);
      else *dst = mk<T>((T)0, (T)0);
    }
    for (int nn = wi; nn < RC; nn += NW) {
      const int n = n0 + nn;
#pragma unroll
      for (int m = 0; m < NT; ++m) {
        const T* tab = (m == 0 ? ict : (m == 1 ? icdt : sdt)) + (size_t)n * cpad + c0;
        T* dst = dM + (nn * NT + m) * CZ;
        for (int cl = lane; cl < CZ; cl += 32) {
          if (n < N && c0 + cl <= chi) async_elem(dst + cl, tab + cl);
          else dst[cl] = (T)0;
        }
      }
    }
    cp_commit();
  };
  for (int c0 = clo; c0 <= chi; c0 += CZ) {
    const int cw = c0 + wi * PG;  // first plane of this warp
    cplx<T> au[PG], av[PG], aw[PG], du[PG], dv[PG];
    T dE[PG], dG[PG], dEt[PG], dGt[PG];
#pragma unroll
    for (int p = 0; p < PG; ++p) {
      au[p] = av[p] = aw[p] = du[p] = dv[p] = mk<T>((T)0, (T)0);
      dE[p] = dG[p] = dEt[p] = dGt[p] = (T)0;
    }
    __syncthreads();  // the previous plane chunk has finished with both slots
    stage(0, c0);
    for (int q = 0; q < nq; ++q) {
      if (q + 1 < nq) {
        stage(q + 1, c0);
        cp_wait_but_newest();
      } else {
        cp_wait_all();
      }
      __syncthreads();  // chunk q (and the amplitudes, node exponentials) visible
      const cplx<T>* Y = sYs + (q & 1) * SLOT_Y;
      const T* Mq = sMs + (q & 1) * SLOT_M;
      const int nend = min(RC, N - q * RC);
      if (cw <= chi) {
        for (int nn = 0; nn < nend; ++nn) {
          const int n = q * RC + nn;
          const cplx<T> yu = Y[(0 * RC + nn) * kLaneK + lane];
          const cplx<T> yv = Y[(1 * RC + nn) * kLaneK + lane];
          const cplx<T> yw = Y[(2 * RC + nn) * kLaneK + lane];
          const T* mr = Mq + nn * NT * CZ + wi * PG;
          T ic[PG];
          ld_row<PG>(mr, ic);
#pragma unroll
          for (int p = 0; p < PG; ++p) {
            au[p].x += ic[p] * yu.x; au[p].y += ic[p] * yu.y;
            av[p].x += ic[p] * yv.x; av[p].y += ic[p] * yv.y;
            aw[p].x += ic[p] * yw.x; aw[p].y += ic[p] * yw.y;
          }
          if (CURL) {
            T id[PG];
            ld_row<PG>(mr + CZ, id);
#pragma unroll
            for (int p = 0; p < PG; ++p) {
              du[p].x += id[p] * yu.x; du[p].y += id[p] * yu.y;
              dv[p].x += id[p] * yv.x; dv[p].y += id[p] * yv.y;
            }
          }
          if (DE) {
            const T en = sE[(size_t)n * kLaneK + lane], gn = sZ[n] * en;
            T sd[PG];
            ld_row<PG>(mr + 2 * CZ, sd);
#pragma unroll
            for (int p = 0; p < PG; ++p) {
              dE[p] += sd[p] * en;
              dG[p] += sd[p] * gn;
            }
            if (CORR == 2) {
              const T et = sE[(size_t)(N - 1 - n) * kLaneK + lane], gt = sZ[N - 1 - n] * et;
#pragma unroll
              for (int p = 0; p < PG; ++p) {
                dEt[p] += sd[p] * et;
                dGt[p] += sd[p] * gt;
              }
            }
          }
        }
      }
      __syncthreads();  // slot q & 1 may be refilled by the next iteration's copies
    }
    if (col < 0 || cw > chi) continue;
#pragma unroll
    for (int p = 0; p < PG; ++p) {
      const int c = cw + p;
      if (c > chi) break;
      const size_t o0 = (size_t)c * plane + col;
      if (kidl < 0) {  // Nyquist column
#pragma unroll
        for (int f = 0; f < (CURL ? 6 : 3); ++f) grid[o0 + f * fstride] = mk<T>((T)0, (T)0);
        continue;
      }
      cplx<T> u = au[p], v = av[p], wv = aw[p], Du = du[p], Dv = dv[p];
      if (CORR) {
        const T zc = sZ[c], ec = sE[(size_t)c * kLaneK + lane];
        auto amp = [&](int q) { return sAmp[q * kLaneK + lane]; };
        u = u + scl(amp(0) + scl(amp(1), zc), ec);
        v = v + scl(amp(4) + scl(amp(5), zc), ec);
        wv = wv + scl(amp(8) + scl(amp(9), zc), ec);
        if (CORR == 2) {
          const T xc = sZ[N - 1 - c], et = sE[(size_t)(N - 1 - c) * kLaneK + lane];
          u = u + scl(amp(2) + scl(amp(3), xc), et);
          v = v + scl(amp(6) + scl(amp(7), xc), et);
          wv = wv + scl(amp(10) + scl(amp(11), xc), et);
        }
        if (DE) {
          Du = Du + scl(amp(0), dE[p]) + scl(amp(1), dG[p]);
          Dv = Dv + scl(amp(4), dE[p]) + scl(amp(5), dG[p]);
          if (CORR == 2) {
            Du = Du + scl(amp(2), dEt[p]) + scl(amp(3), dGt[p]);
            Dv = Dv + scl(amp(6), dEt[p]) + scl(amp(7), dGt[p]);
          }
        }
      }
      grid[o0] = scl(u, scale);
      grid[o0 + fstride] = scl(v, scale);
      grid[o0 + 2 * fstride] = scl(wv, scale);
      if (CURL) {
        // omega = 1/2 (i ky w - Dv, Du - i kx w, i kx v - i ky u)
        const cplx<T> ox = scl(mul_i(wv), hky) - scl(Dv, (T)0.5);
        const cplx<T> oy = scl(Du, (T)0.5) - scl(mul_i(wv), hkx);
        const cplx<T> oz = scl(mul_i(v), hkx) - scl(mul_i(u), hky);
        grid[o0 + 3 * fstride] = scl(ox, scale);
        grid[o0 + 4 * fstride] = scl(oy, scale);
        grid[o0 + 5 * fstride] = scl(oz, scale);
      }
    }
  }
  cp_wait_all();  // no copy outlives the block when no plane is occupied
}

template <typename T> constexpr int fwd_nb() { return sizeof(T) == 4 ? 24 : 12; }
template <typename T> constexpr int bwd_cb() { return sizeof(T) == 4 ? 12 : 4; }

size_t fwd_smem(const Plan& p, size_t tsz) { return 2 * (size_t)p.g.nz * p.kt.npad * tsz; }
size_t bwd_smem(const Plan& p, size_t tsz) { return (p.g.spectral_curl ? 3 : 1) * (size_t)p.g.nz * p.kt.cpad * tsz; }

// launch shape of the lane-per-wavenumber forward transform; threads = 0 when it does not apply
struct LaneCfg {
  int threads = 0, cz = 0;
  size_t smem = 0;
  int pg = 0;  // forward transform: Chebyshev rows per warp (fwd_pg or fwd_pg_wide)
};
constexpr int kFwdPlanes = 8;                // planes per double-buffered chunk of the forward transform
constexpr size_t kBwdLaneSmem = 200 * 1024;  // largest backward stage

template <typename T>
LaneCfg fwd_lane_cfg(const Geometry& g) {
  LaneCfg c;
  int PG = fwd_pg<T>();
  int nw = (g.nz + PG - 1) / PG;
  if (32 * nw > fwd_max_threads<T>()) {
    PG = fwd_pg_wide<T>();
    nw = (g.nz + PG - 1) / PG;
  }
  if (g.nz > 128 || 32 * nw > fwd_max_threads<T>()) return c;
  const int nf = g.spectral_curl ? 6 : 3;
  const size_t per_plane = (size_t)nf * kLaneK * sizeof(cplx<T>) + (size_t)2 * nw * PG * sizeof(T);
  c.pg = PG;
  c.threads = 32 * nw;
  c.cz = std::min(g.nz, kFwdPlanes);      // planes per pipelined chunk
  c.smem = 2 * per_plane * (size_t)c.cz;  // two slots
  return c;
}

template <typename T>
size_t bwd_lane_smem(const Geometry& g) {
  const size_t N = (size_t)g.nz, N4 = (N + 3) & ~(size_t)3;
  const bool corr = g.mode != DPS_FREE;
  const size_t nt = g.spectral_curl ? (corr ? 3 : 2) : 1;
  const size_t cz = (size_t)bwd_warps<T>() * bwd_pg<T>();
  size_t b = 2 * (3 * (size_t)kBwdRows * kLaneK * sizeof(cplx<T>) + (size_t)kBwdRows * nt * cz * sizeof(T));
  if (corr) b += 12 * kLaneK * sizeof(cplx<T>) + N * kLaneK * sizeof(T) + N4 * sizeof(T);
  return (g.nz <= 128 && b <= kBwdLaneSmem) ? b : 0;
}

template <typename T, bool CURL, int CORR>
void launch_bwd_lane(const Plan& p, int kx0, int w, cudaStream_t s) {
  const Geometry& g = p.g;
  const unsigned blocks = (unsigned)(((int64_t)w * g.ny + kLaneK - 1) / kLaneK);
  bwd_lane_kernel<T, bwd_pg<T>(), CURL, CORR><<<blocks, 32 * bwd_warps<T>(), bwd_lane_smem<T>(g), s>>>(
      g, reinterpret_cast<const T*>(p.kt.ict), reinterpret_cast<const T*>(p.kt.icdt),
      reinterpret_cast<const T*>(p.kt.sdt), p.kt.cpad, reinterpret_cast<const T*>(p.tab.zeta),
      reinterpret_cast<const cplx<T>*>(p.kt.kbuf), reinterpret_cast<const cplx<T>*>(p.kt.kaux),
      reinterpret_cast<cplx<T>*>(p.grid), p.zrange, kx0, w);
}

template <typename T, bool CURL, int CORR>
bool set_bwd_lane_smem(size_t bytes) {
  return bytes == 0 || allow_smem(bwd_lane_kernel<T, bwd_pg<T>(), CURL, CORR>);
}

}  // namespace

template <typename T>
size_t bvp_slot_bytes(const Plan& p) {
  const size_t N = (size_t)p.g.nz;
  return 3 * N * sizeof(cplx<double>) + 3 * N * sizeof(double) + N * sizeof(cplx<T>);
}

template <typename T>
int bvp_occupancy_blocks(const Plan& p) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_kernel<T, false>, kBvpThreads, 0);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 4) per_sm = 4;
  return per_sm * sms;
}

template <typename T>
int bvp_prepare(Plan& p) {
  // shared-memory staging of the transform tables of the per-thread fallbacks when they fit
  const size_t fs = fwd_smem(p, sizeof(T)), bs = bwd_smem(p, sizeof(T));
  p.kt.fwd_smem = fs <= 160 * 1024 ? (int)fs : 0;
  p.kt.bwd_smem = bs <= 160 * 1024 ? (int)bs : 0;
  constexpr int NB = fwd_nb<T>(), CB = bwd_cb<T>();
  if (!allow_smem(fwd_kernel<T, NB>) || !allow_smem(bwd_kernel<T, CB, true>) || !allow_smem(bwd_kernel<T, CB, false>))
    return 0;
  const LaneCfg fc = fwd_lane_cfg<T>(p.g);
  if (fc.threads > 0) {
    constexpr int PG = fwd_pg<T>(), PW = fwd_pg_wide<T>();
    if (!allow_smem(fwd_lane_kernel<T, PG, true>) || !allow_smem(fwd_lane_kernel<T, PG, false>) ||
        !allow_smem(fwd_lane_kernel<T, PW, true>) || !allow_smem(fwd_lane_kernel<T, PW, false>))
      return 0;
    if constexpr (sizeof(T) == 4) {
      if (!allow_smem(fwd_lane_kernel<T, PG, true, 3>)) return 0;
    }
  }
  const size_t bl = bwd_lane_smem<T>(p.g);
  if (bl > 0) {
    if (!set_bwd_lane_smem<T, true, 0>(bl) || !set_bwd_lane_smem<T, true, 1>(bl) ||
        !set_bwd_lane_smem<T, true, 2>(bl) || !set_bwd_lane_smem<T, false, 0>(bl) ||
        !set_bwd_lane_smem<T, false, 1>(bl) || !set_bwd_lane_smem<T, false, 2>(bl))
      return 0;
  }
  return 1;
}

template <typename T>
void launch_bvp(const Plan& p, int part, int kx0, int w, cudaStream_t s) {
  const Geometry& g = p.g;
  const int64_t total = (int64_t)w * g.ny;
  const unsigned blocks = (unsigned)((total + kBvpThreads - 1) / kBvpThreads);
  constexpr int NB = fwd_nb<T>(), CB = bwd_cb<T>();
  cplx<T>* grid = reinterpret_cast<cplx<T>*>(p.grid);
  cplx<T>* kbuf = reinterpret_cast<cplx<T>*>(p.kt.kbuf);
  cplx<T>* kaux = reinterpret_cast<cplx<T>*>(p.kt.kaux);
  const LaneCfg fc = fwd_lane_cfg<T>(g);
  if (part == 0 && sizeof(T) == 4 && p.cheb_tc) {
    launch_cheb_fwd_tc(p, kx0, w, s);
  } else if (part == 0 && fc.threads > 0) {
    const unsigned lb = (unsigned)((total + kLaneK - 1) / kLaneK);
    constexpr int PG = fwd_pg<T>(), PW = fwd_pg_wide<T>();
    const T* ct = reinterpret_cast<const T*>(p.kt.ct);
    const T* dct = reinterpret_cast<const T*>(p.kt.dct);
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      // the six-field (spectral-curl) form only: the three-field form fits three blocks per SM as it
      // is (70 registers) and measured slower compact (5.20 -> 5.30 ms on rollers_1m)
      if (fc.pg == PG && fc.threads <= kFwdCompactThreads && g.spectral_curl) {
        fwd_lane_kernel<T, PG, true, 3><<<lb, fc.threads, fc.smem, s>>>(g, ct, dct, p.kt.npad, grid, kbuf, p.zrange,
                                                                        kx0, w, fc.cz);
        done = true;
      }
    }
    if (done) {
    } else if (fc.pg == PG) {
      if (g.spectral_curl)
        fwd_lane_kernel<T, PG, true><<<lb, fc.threads, fc.smem, s>>>(g, ct, dct, p.kt.npad, grid, kbuf, p.zrange, kx0,
                                                                     w, fc.cz);
      else
        fwd_lane_kernel<T, PG, false><<<lb, fc.threads, fc.smem, s>>>(g, ct, dct, p.kt.npad, grid, kbuf, p.zrange, kx0,
                                                                      w, fc.cz);
    } else {
      if (g.spectral_curl)
        fwd_lane_kernel<T, PW, true><<<lb, fc.threads, fc.smem, s>>>(g, ct, dct, p.kt.npad, grid, kbuf, p.zrange, kx0,
                                                                     w, fc.cz);
      else
        fwd_lane_kernel<T, PW, false><<<lb, fc.threads, fc.smem, s>>>(g, ct, dct, p.kt.npad, grid, kbuf, p.zrange, kx0,
                                                                      w, fc.cz);
    }
  } else if (part == 2 && sizeof(T) == 4 && p.cheb_tc_bwd) {
    launch_cheb_bwd_tc(p, kx0, w, s);
  } else if (part == 2 && bwd_lane_smem<T>(g) > 0) {
    const int corr = g.mode == DPS_FREE ? 0 : (g.mode == DPS_SLIT ? 2 : 1);
    if (g.spectral_curl) {
      if (corr == 0) launch_bwd_lane<T, true, 0>(p, kx0, w, s);
      else if (corr == 1) launch_bwd_lane<T, true, 1>(p, kx0, w, s);
      else launch_bwd_lane<T, true, 2>(p, kx0, w, s);
    } else {
      if (corr == 0) launch_bwd_lane<T, false, 0>(p, kx0, w, s);
      else if (corr == 1) launch_bwd_lane<T, false, 1>(p, kx0, w, s);
      else launch_bwd_lane<T, false, 2>(p, kx0, w, s);
    }
  } else if (part == 0) {
    fwd_kernel<T, NB><<<blocks, kBvpThreads, p.kt.fwd_smem, s>>>(
        g, reinterpret_cast<const T*>(p.kt.ct), reinterpret_cast<const T*>(p.kt.dct), p.kt.npad, p.kt.fwd_smem > 0,
        grid, kbuf, p.zrange, kx0, w);
  } else if (part == 1) {
    const size_t N = (size_t)g.nz;
    const size_t slots = (size_t)p.bvp_blocks * kBvpThreads;
    unsigned char* base = reinterpret_cast<unsigned char*>(p.ws);
    cplx<double>* sw = reinterpret_cast<cplx<double>*>(base);
    double* fr = reinterpret_cast<double*>(base + 3 * N * slots * sizeof(cplx<double>));
    cplx<T>* pws = reinterpret_cast<cplx<T>*>(base + 3 * N * slots * (sizeof(cplx<double>) + sizeof(double)));
    const T* bandT = reinterpret_cast<const T*>(p.kt.bandT);
    const double tpx = 2.0 * M_PI / g.Lx, tpy = 2.0 * M_PI / g.Ly;  // host divisions
    if (p.kt.fac && g.slip)
      solve_tab_kernel<T, true><<<p.bvp_blocks, kBvpThreads, 0, s>>>(g, p.tab.band, bandT, p.kt.fac, p.kt.KP, kbuf, kaux,
                                                                    pws, sw, kx0, w, tpx, tpy);
    else if (p.kt.fac)
      solve_tab_kernel<T, false><<<p.bvp_blocks, kBvpThreads, 0, s>>>(g, p.tab.band, bandT, p.kt.fac, p.kt.KP, kbuf,
                                                                     kaux, pws, sw, kx0, w, tpx, tpy);
    else if (g.slip)
      solve_kernel<T, true><<<p.bvp_blocks, kBvpThreads, 0, s>>>(g, p.tab.band, reinterpret_cast<const T*>(p.kt.bandT),
                                                                 kbuf, kaux, pws, sw, fr, kx0, w);
    else
      solve_kernel<T, false><<<p.bvp_blocks, kBvpThreads, 0, s>>>(g, p.tab.band, reinterpret_cast<const T*>(p.kt.bandT),
                                                                  kbuf, kaux, pws, sw, fr, kx0, w);
  } else if (g.spectral_curl) {
    bwd_kernel<T, CB, true><<<blocks, kBvpThreads, p.kt.bwd_smem, s>>>(
        g, reinterpret_cast<const T*>(p.kt.ict), reinterpret_cast<const T*>(p.kt.icdt),
        reinterpret_cast<const T*>(p.kt.sdt), reinterpret_cast<const T*>(p.tab.zeta), p.kt.cpad, p.kt.bwd_smem > 0, kbuf,
        kaux, grid, p.zrange, kx0, w);
  } else {
    bwd_kernel<T, CB, false><<<blocks, kBvpThreads, p.kt.bwd_smem, s>>>(
        g, reinterpret_cast<const T*>(p.kt.ict), nullptr, nullptr, reinterpret_cast<const T*>(p.tab.zeta), p.kt.cpad,
        p.kt.bwd_smem > 0, kbuf, kaux, grid, p.zrange, kx0, w);
  }
}

dps_status bvp_factor_table(Plan& p) {
  const Geometry& g = p.g;
  const int64_t KP = (int64_t)g.nkx * (g.ny / 2 + 1);
  const size_t bytes = (size_t)KP * g.nz * 4 * sizeof(double);
  void* q = nullptr;
  if (cudaMalloc(&q, bytes) != cudaSuccess) {
    cudaGetLastError();
    return DPS_ERR_OOM;
  }
  p.kt.fac = reinterpret_cast<double*>(q);
  p.kt.KP = KP;
  p.device_bytes += (int64_t)bytes;
  factor_kernel<<<(unsigned)((KP + 127) / 128), 128>>>(g, p.tab.band, p.kt.fac, KP);
  return cudaGetLastError() == cudaSuccess ? DPS_OK : DPS_ERR_CUDA;
}

template size_t bvp_slot_bytes<float>(const Plan&);
template size_t bvp_slot_bytes<double>(const Plan&);
template int bvp_occupancy_blocks<float>(const Plan&);
template int bvp_occupancy_blocks<double>(const Plan&);
template int bvp_prepare<float>(Plan&);
template int bvp_prepare<double>(Plan&);
template void launch_bvp<float>(const Plan&, int, int, int, cudaStream_t);
template void launch_bvp<double>(const Plan&, int, int, int, cudaStream_t);

}  // namespace dps
