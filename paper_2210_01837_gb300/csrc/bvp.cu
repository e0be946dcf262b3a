// Per-wavenumber stage of the doubly-periodic Stokes solve (steps 2-7 of Sec. III.D, z part).
//
// One thread owns one (kx, ky) of the half spectrum for the whole stage (persistent grid; each
// thread keeps a private workspace slot laid out [array][row][slot] so that the per-row accesses
// of a warp are coalesced):
//   A. Chebyshev coefficients of the three force components by DCT-I of the occupied planes, with
//      the half-curl of the torque field added in Fourier-Chebyshev space (Eq. 7).
//   B. DP pressure BVP (Eqs. 15, 17), FP64.
//   C. DP velocity BVPs (Eqs. 18, 22, 24), three right-hand sides sharing the factorisation, FP64.
//   D. Wall correction: boundary values of the DP velocity by direct summation, correction
//      amplitudes in FP64 (bottom wall: Eqs. 41-44; slit: Eqs. A4-A10 with zero slip, solved in
//      closed form), the correction added as Chebyshev coefficients of its node values (step 6).
//   E. Curl (Eq. 11) in Fourier-Chebyshev space.
//   F. Inverse DCT-I to the occupied planes, times 1/(Nx Ny) for the inverse xy transform.
// k = 0 follows Sec. III.C (Eqs. 47-52; Eq. A12); Nyquist modes are set to zero.
//
// BVP discretisation (the paper defers it to Greengard's spectral integration): s in [-1, 1],
// y = trunc_N(B B c) + a0 T0 + a1 T1 with c the coefficients of y_ss; rows
// (2/H)^2 c_n - k^2 y_n = r_n, n = 0..N-1, plus two boundary rows.  B B couples c_{n-2}, c_n,
// c_{n+2} only (coefficients l_n, d_n, u_n), so the system splits into an even and an odd
// tridiagonal system, each bordered by one unknown (a0 or a1, row 0 or 1 only) and by one dense
// boundary row; the Dirichlet-to-Neumann rows combine into one row per parity.  Each parity is
// eliminated from the last row down (c_n = s_n - t_n c_{n-2}), folding the boundary row as it
// goes, which leaves a 2x2 system for (c_par, a_par); the rows are diagonally dominant, so no
// pivoting is needed.  The factorisation depends on |k| only and is shared by all four solves.
#include <math.h>

#include "dps_internal.cuh"

namespace dps {

namespace {

struct BvpTabs {
  const double* band;   // l, d, u, P, Q  each [N]
  const void* dct;      // C[n][c]
  const void* dctd;     // (2/H) D C
  const void* idct;     // IC[c][n]
  const void* zeta;     // z_c - zmin
};

template <typename T>
struct Ws {
  cplx<T>* wt;          // [7][N][slots]: coef u,v,w | omega x,y,z | pressure
  cplx<double>* wd;     // [3][N][slots]: sweep values for up to three right-hand sides
  double* wr;           // [3][N][slots]: rho, t, folded boundary coefficient
  int N, slots, slot;
  __device__ __forceinline__ cplx<T>& co(int a, int n) const { return wt[((size_t)a * N + n) * slots + slot]; }
  __device__ __forceinline__ cplx<double>& sw(int a, int n) const { return wd[((size_t)a * N + n) * slots + slot]; }
  __device__ __forceinline__ double& fr(int a, int n) const { return wr[((size_t)a * N + n) * slots + slot]; }
};

template <typename T> __device__ __forceinline__ cplx<double> up(cplx<T> a) { return mk<double>((double)a.x, (double)a.y); }
template <typename T> __device__ __forceinline__ cplx<T> down(cplx<double> a) { return mk<T>((T)a.x, (T)a.y); }

__device__ __forceinline__ cplx<double> cdiv(cplx<double> a, cplx<double> b) {
  const double den = b.x * b.x + b.y * b.y;
  return mk<double>((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

template <typename T> __device__ __forceinline__ T ld(const void* p, int i) { return __ldg(reinterpret_cast<const T*>(p) + i); }

template <typename T>
__device__ __forceinline__ cplx<T> gld(const cplx<T>* grid, size_t off) { return grid[off]; }

// ---------------------------------------------------------------------------------------------
template <typename T, int NCH>
__device__ void solve_one(const Geometry& g, const BvpTabs& tb, cplx<T>* __restrict__ grid, const int clo,
                          const int chi, const int64_t kidx, const Ws<T>& ws) {
  const int N = g.nz;
  const int kxi = (int)(kidx % g.nkx);
  const int kyi = (int)(kidx / g.nkx);
  const size_t plane = (size_t)g.ny * g.pitch;
  const size_t col = (size_t)kyi * g.pitch + kxi;
  auto gaddr = [&](int f, int c) -> size_t { return ((size_t)f * g.nz + c) * plane + col; };
  const int nfo = g.nfields;  // output fields (3 velocity [+ 3 half-curl])
  const bool nyq = ((g.nx % 2 == 0) && kxi == g.nx / 2) || ((g.ny % 2 == 0) && kyi == g.ny / 2);
  if (nyq) {
    for (int f = 0; f < nfo; ++f)
      for (int c = clo; c <= chi; ++c) grid[gaddr(f, c)] = mk<T>((T)0, (T)0);
    return;
  }
  const int nyv = (kyi < (g.ny + 1) / 2) ? kyi : kyi - g.ny;
  const double kx = 2.0 * M_PI * (double)kxi / g.Lx;
  const double ky = 2.0 * M_PI * (double)nyv / g.Ly;
  const double kk = sqrt(kx * kx + ky * ky);
  const double sH = 2.0 / g.H;         // d/dz = (2/H) d/ds
  const double sig = sH * sH;
  const double kap = kk * kk;
  const double inv_eta = 1.0 / g.eta;
  const double* bl = tb.band;
  const double* bd = tb.band + N;
  const double* bu = tb.band + 2 * N;
  const double* bP = tb.band + 3 * N;
  const double* bQ = tb.band + 4 * N;

  // ---------------- A. forward DCT-I with the half-curl source ----------------------------------
  {
    const T hkx = (T)(0.5 * kx), hky = (T)(0.5 * ky);
    for (int o = 0; o < 3; ++o) {
      for (int n0 = 0; n0 < N; n0 += NCH) {
        cplx<T> acc[NCH];
#pragma unroll
        for (int j = 0; j < NCH; ++j) acc[j] = mk<T>((T)0, (T)0);
        for (int c = clo; c <= chi; ++c) {
          cplx<T> a = gld(grid, gaddr(o, c));
          cplx<T> b = mk<T>((T)0, (T)0);
          if (g.with_torque) {
            if (o == 0) {        // Fx + 1/2 i ky tz ;  - 1/2 D ty
              a = a + mul_i(scl(gld(grid, gaddr(5, c)), hky));
              b = scl(gld(grid, gaddr(4, c)), (T)-0.5);
            } else if (o == 1) { // Fy - 1/2 i kx tz ;  + 1/2 D tx
              a = a - mul_i(scl(gld(grid, gaddr(5, c)), hkx));
              b = scl(gld(grid, gaddr(3, c)), (T)0.5);
            } else {             // Fz + 1/2 (i kx ty - i ky tx)
              a = a + mul_i(scl(gld(grid, gaddr(4, c)), hkx) - scl(gld(grid, gaddr(3, c)), hky));
            }
          }
#pragma unroll
          for (int j = 0; j < NCH; ++j) {
            const int n = n0 + j;
            if (n < N) {
              const T cm = ld<T>(tb.dct, n * N + c);
              acc[j].x += cm * a.x;
              acc[j].y += cm * a.y;
              if (g.with_torque && o < 2) {
                const T dm = ld<T>(tb.dctd, n * N + c);
                acc[j].x += dm * b.x;
                acc[j].y += dm * b.y;
              }
            }
          }
        }
#pragma unroll
        for (int j = 0; j < NCH; ++j)
          if (n0 + j < N) ws.co(o, n0 + j) = acc[j];
      }
    }
  }

  if (kxi == 0 && kyi == 0) {
    // ---------------- k = 0 (Sec. III.C; Appendix A.2) -------------------------------------------
    for (int o = 0; o < 3; ++o) {
      if (g.mode == DPS_FREE || o == 2) {
        for (int n = 0; n < N; ++n) ws.co(o, n) = mk<T>((T)0, (T)0);
        continue;
      }
      // sigma c_n = -f_n / eta ; y = B B c + a0 + a1 s with the two boundary rows
      cplx<double> Sp = mk<double>(0, 0), Sm = mk<double>(0, 0), Pd = mk<double>(0, 0);
      for (int n = 0; n < N; ++n) {
        const cplx<double> cn = scl(up(ws.co(o, n)), -inv_eta / sig);
        const double sgn = (n & 1) ? -1.0 : 1.0;
        Sp = Sp + scl(cn, bQ[n]);
        Sm = Sm + scl(cn, sgn * bQ[n]);
        Pd = Pd + scl(cn, bP[n]);
      }
      cplx<double> a0, a1;
      if (g.mode == DPS_BOTTOM_WALL) {  // y(-1) = 0, y_s(+1) = 0
        a1 = scl(Pd, -1.0);
        a0 = a1 - Sm;
      } else {                           // y(-1) = y(+1) = 0
        a0 = scl(Sp + Sm, -0.5);
        a1 = scl(Sp - Sm, -0.5);
      }
      // y_n = l_n c_{n-2} + d_n c_n + u_n c_{n+2} (+ a0, a1): stage c in the sweep area first
      for (int n = 0; n < N; ++n) ws.sw(0, n) = scl(up(ws.co(o, n)), -inv_eta / sig);
      for (int n = 0; n < N; ++n) {
        cplx<double> y = scl(ws.sw(0, n), bd[n]);
        if (n >= 2) y = y + scl(ws.sw(0, n - 2), bl[n]);
        if (n + 2 < N) y = y + scl(ws.sw(0, n + 2), bu[n]);
        if (n == 0) y = y + a0;
        if (n == 1) y = y + a1;
        ws.co(o, n) = down<T>(y);
      }
    }
  } else {
    // ---------------- B. pressure: (D^2 - k^2) p = i kx f + i ky g + D h --------------------------
    cplx<double> ptop = mk<double>(0, 0), pbot = mk<double>(0, 0);
    for (int par = 0; par < 2; ++par) {
      const int nlast = ((N - 1 - par) & 1) ? N - 2 : N - 1;  // largest n < N with n = par (mod 2)
      cplx<double> s_next = mk<double>(0, 0);
      double t_next = 0.0;
      double bfold = 0.0;              // folded boundary-row coefficient on the current c_n
      cplx<double> gacc = mk<double>(0, 0);
      // derivative recurrence of h over the opposite parity: b_n = b_{n+2} + 2(n+1) h_{n+1}
      cplx<double> dh_next = mk<double>(0, 0);
      for (int n = nlast; n >= par; n -= 2) {
        cplx<double> dh = dh_next;
        if (n + 1 < N) dh = dh + scl(up(ws.co(2, n + 1)), 2.0 * (n + 1));
        dh_next = dh;
        if (n == 0) dh = scl(dh, 0.5);
        const cplx<double> f = up(ws.co(0, n)), gg = up(ws.co(1, n));
        const cplx<double> r = mk<double>(-kx * f.y - ky * gg.y + sH * dh.x, kx * f.x + ky * gg.x + sH * dh.y);
        const double U = -kap * bu[n];
        const double beta_n = sH * bP[n] + kk * bQ[n];
        const double bcur = (n == nlast) ? beta_n : bfold;
        if (n > par) {
          const double rho = 1.0 / ((sig - kap * bd[n]) - U * t_next);
          const double t = rho * (-kap * bl[n]);
          const cplx<double> s = scl(r - scl(s_next, U), rho);
          ws.fr(0, n) = rho;
          ws.fr(1, n) = t;
          ws.fr(2, n) = bcur;
          ws.sw(0, n) = s;
          gacc = gacc - scl(s, bcur);
          bfold = bP[n - 2] * sH + kk * bQ[n - 2] - bcur * t;
          s_next = s;
          t_next = t;
        } else {
          // row `par`: D'_par c_par - kappa a_par = r_par - U s_{par+2} ; boundary: beta_a a + bcur c = g'
          const double Dp = (sig - kap * bd[n]) - U * t_next;
          const double beta_a = (par == 0) ? kk : (sH + kk);
          const cplx<double> rhs = r - scl(s_next, U);
          const double det = Dp * beta_a + kap * bcur;
          const cplx<double> c0 = scl(scl(rhs, beta_a) + scl(gacc, kap), 1.0 / det);
          const cplx<double> a = scl(scl(gacc, Dp) - scl(rhs, bcur), 1.0 / det);
          ws.fr(0, n) = Dp;
          ws.fr(1, n) = 0.0;
          ws.fr(2, n) = bcur;
          // ascending substitution, boundary sums, y = B B c + a
          cplx<double> cm2 = mk<double>(0, 0), cm = c0;  // c_{n-2}, c_n
          const double sgn = par ? -1.0 : 1.0;
          cplx<double> sp = scl(c0, bQ[par]);
          for (int m = par + 2; m <= nlast + 2; m += 2) {
            cplx<double> cnew = mk<double>(0, 0);
            if (m <= nlast) {
              cnew = ws.sw(0, m) - scl(cm, ws.fr(1, m));
              sp = sp + scl(cnew, bQ[m]);
            }
            // finish y_{m-2} = l c_{m-4} + d c_{m-2} + u c_m
            const int q = m - 2;
            cplx<double> y = scl(cm, bd[q]) + scl(cnew, bu[q]);
            if (q >= 2) y = y + scl(cm2, bl[q]);
            if (q == par) y = y + a;
            ws.co(6, q) = down<T>(y);
            cm2 = cm;
            cm = cnew;
          }
          ptop = ptop + sp + a;
          pbot = pbot + scl(sp, sgn) + scl(a, sgn);
        }
      }
    }

    // ---------------- C. velocity: three right-hand sides, shared factorisation ------------------
    const cplx<double> ik_top = scl(ptop, 1.0 / (2.0 * kk * g.eta));
    const cplx<double> ik_bot = scl(pbot, 1.0 / (2.0 * kk * g.eta));
    // boundary data (g_top, g_bot) per field: u, v use -+ i k p/(2 k eta), w uses p/(2 eta)
    cplx<double> gt[3], gb[3];
    gt[0] = scl(mul_i(ik_top), -kx);
    gb[0] = scl(mul_i(ik_bot), kx);
    gt[1] = scl(mul_i(ik_top), -ky);
    gb[1] = scl(mul_i(ik_bot), ky);
    gt[2] = scl(ptop, 0.5 * inv_eta);
    gb[2] = scl(pbot, 0.5 * inv_eta);
    cplx<double> vtop[3], vbot[3];
    for (int f = 0; f < 3; ++f) { vtop[f] = mk<double>(0, 0); vbot[f] = mk<double>(0, 0); }
    for (int par = 0; par < 2; ++par) {
      const int nlast = ((N - 1 - par) & 1) ? N - 2 : N - 1;
      cplx<double> s_next[3], gacc[3];
      for (int f = 0; f < 3; ++f) {
        s_next[f] = mk<double>(0, 0);
        gacc[f] = par ? scl(gt[f] + gb[f], 0.5) : scl(gt[f] - gb[f], 0.5);
      }
      cplx<double> dp_next = mk<double>(0, 0);
      for (int n = nlast; n >= par; n -= 2) {
        cplx<double> dp = dp_next;
        if (n + 1 < N) dp = dp + scl(up(ws.co(6, n + 1)), 2.0 * (n + 1));
        dp_next = dp;
        if (n == 0) dp = scl(dp, 0.5);
        const cplx<double> pn = up(ws.co(6, n));
        cplx<double> r[3];
        const cplx<double> f0 = up(ws.co(0, n)), f1 = up(ws.co(1, n)), f2 = up(ws.co(2, n));
        r[0] = scl(scl(mul_i(pn), kx) - f0, inv_eta);
        r[1] = scl(scl(mul_i(pn), ky) - f1, inv_eta);
        r[2] = scl(scl(dp, sH) - f2, inv_eta);
        const double U = -kap * bu[n];
        const double bcur = ws.fr(2, n);
        if (n > par) {
          const double rho = ws.fr(0, n);
          for (int f = 0; f < 3; ++f) {
            const cplx<double> s = scl(r[f] - scl(s_next[f], U), rho);
            ws.sw(f, n) = s;
            gacc[f] = gacc[f] - scl(s, bcur);
            s_next[f] = s;
          }
        } else {
          const double Dp = ws.fr(0, n);
          const double beta_a = (par == 0) ? kk : (sH + kk);
          const double det = Dp * beta_a + kap * bcur;
          const double sgn = par ? -1.0 : 1.0;
          for (int f = 0; f < 3; ++f) {
            const cplx<double> rhs = r[f] - scl(s_next[f], U);
            const cplx<double> c0 = scl(scl(rhs, beta_a) + scl(gacc[f], kap), 1.0 / det);
            const cplx<double> a = scl(scl(gacc[f], Dp) - scl(rhs, bcur), 1.0 / det);
            cplx<double> cm2 = mk<double>(0, 0), cm = c0;
            cplx<double> sp = scl(c0, bQ[par]);
            for (int m = par + 2; m <= nlast + 2; m += 2) {
              cplx<double> cnew = mk<double>(0, 0);
              if (m <= nlast) {
                cnew = ws.sw(f, m) - scl(cm, ws.fr(1, m));
                sp = sp + scl(cnew, bQ[m]);
              }
              const int q = m - 2;
              cplx<double> y = scl(cm, bd[q]) + scl(cnew, bu[q]);
              if (q >= 2) y = y + scl(cm2, bl[q]);
              if (q == par) y = y + a;
              ws.co(f, q) = down<T>(y);
              cm2 = cm;
              cm = cnew;
            }
            vtop[f] = vtop[f] + sp + a;
            vbot[f] = vbot[f] + scl(sp, sgn) + scl(a, sgn);
          }
        }
      }
    }

    // ---------------- D. wall correction ---------------------------------------------------------
    if (g.mode != DPS_FREE) {
      // wall data: minus the DP velocity at the wall(s); tangential parts along k (L) and across (T)
      const double ex = kx / kk, ey = ky / kk;
      auto Lp = [&](cplx<double> u, cplx<double> v) { return scl(u, ex) + scl(v, ey); };
      auto Tp = [&](cplx<double> u, cplx<double> v) { return scl(v, ex) - scl(u, ey); };
      const cplx<double> u0L = scl(Lp(vbot[0], vbot[1]), -1.0), u0T = scl(Tp(vbot[0], vbot[1]), -1.0);
      const cplx<double> w0 = scl(vbot[2], -1.0);
      cplx<double> AL = u0L, Az = w0, AT = u0T;
      cplx<double> BL = mk<double>(0, 0), Bz = mk<double>(0, 0), BT = mk<double>(0, 0);
      if (g.mode == DPS_SLIT) {
        const cplx<double> uHL = scl(Lp(vtop[0], vtop[1]), -1.0), uHT = scl(Tp(vtop[0], vtop[1]), -1.0);
        const cplx<double> wH = scl(vtop[2], -1.0);
        const double kH = kk * g.H;
        const double E = exp(-kH);
        const double E2 = E * E;
        // transverse: [1 E; E 1] [AT; BT] = [u0T; uHT]
        AT = scl(u0T - scl(uHT, E), 1.0 / (1.0 - E2));
        BT = scl(uHT - scl(u0T, E), 1.0 / (1.0 - E2));
        // longitudinal/normal: A = a0 - E M1 B, B = b0 - E M2 A  =>  (I - E^2 M1 M2) A = a0 - E M1 b0
        // M1 = [[1-kH, i kH],[i kH, 1+kH]], M2 = [[1-kH, -i kH],[-i kH, 1+kH]]
        const double k2H2 = kH * kH;
        const cplx<double> m11 = mk<double>(1.0 - E2 * (1.0 - 2.0 * kH + 2.0 * k2H2), 0.0);
        const cplx<double> m12 = mk<double>(0.0, -E2 * 2.0 * k2H2);
        const cplx<double> m21 = mk<double>(0.0, E2 * 2.0 * k2H2);
        const cplx<double> m22 = mk<double>(1.0 - E2 * (1.0 + 2.0 * kH + 2.0 * k2H2), 0.0);
        // M1 b0
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
      // pressure amplitudes / (2 eta): bottom pi_b = k (Az - i AL), top pi_t = -k (Bz + i BL)
      const cplx<double> pib = scl(Az - mul_i(AL), kk);
      const cplx<double> pit = scl(Bz + mul_i(BL), -kk);
      // coefficient of E_n, G_n (bottom family) and (-1)^n E_n, (-1)^n G_n (top family)
      // u_L = (AL - i pi_b zeta) e^{-k zeta} + (BL - i pi_t xi) e^{-k xi}
      // w   = (Az + pi_b zeta) e^{-k zeta} + (Bz - pi_t xi) e^{-k xi},  u_T = AT e + BT e
      cplx<double> cE[3], cG[3], tE[3], tG[3];
      const cplx<double> gbL = scl(mul_i(pib), -1.0), gtL = scl(mul_i(pit), -1.0);
      cE[0] = scl(AL, ex) - scl(AT, ey);  cG[0] = scl(gbL, ex);
      tE[0] = scl(BL, ex) - scl(BT, ey);  tG[0] = scl(gtL, ex);
      cE[1] = scl(AL, ey) + scl(AT, ex);  cG[1] = scl(gbL, ey);
      tE[1] = scl(BL, ey) + scl(BT, ex);  tG[1] = scl(gtL, ey);
      cE[2] = Az;                          cG[2] = pib;
      tE[2] = Bz;                          tG[2] = scl(pit, -1.0);
      cplx<T> ce[3], cg[3], te[3], tg[3];
      for (int f = 0; f < 3; ++f) { ce[f] = down<T>(cE[f]); cg[f] = down<T>(cG[f]); te[f] = down<T>(tE[f]); tg[f] = down<T>(tG[f]); }
      const T kt = (T)kk;
      for (int n0 = 0; n0 < N; n0 += NCH) {
        T aE[NCH], aG[NCH];
#pragma unroll
        for (int j = 0; j < NCH; ++j) { aE[j] = (T)0; aG[j] = (T)0; }
        for (int c = 0; c < N; ++c) {
          const T zt = ld<T>(tb.zeta, c);
          const T e = (sizeof(T) == 4) ? (T)expf((float)(-kt * zt)) : (T)exp((double)(-kt * zt));
          const T ze = zt * e;
#pragma unroll
          for (int j = 0; j < NCH; ++j) {
            if (n0 + j < N) {
              const T cm = ld<T>(tb.dct, (n0 + j) * N + c);
              aE[j] += cm * e;
              aG[j] += cm * ze;
            }
          }
        }
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
          const int n = n0 + j;
          if (n < N) {
            const T sg = (n & 1) ? (T)-1 : (T)1;
            for (int f = 0; f < 3; ++f) {
              cplx<T> v = ws.co(f, n);
              v = v + scl(ce[f], aE[j]) + scl(cg[f], aG[j]);
              if (g.mode == DPS_SLIT) v = v + scl(scl(te[f], aE[j]) + scl(tg[f], aG[j]), sg);
              ws.co(f, n) = v;
            }
          }
        }
      }
    }
  }

  // ---------------- E. half-curl omega = 1/2 curl u -----------------------------------------------
  if (g.with_torque) {
    const T hkx = (T)(0.5 * kx), hky = (T)(0.5 * ky), hs = (T)(0.5 * sH);
    // descending derivative recurrences for u and v (b_n = b_{n+2} + 2(n+1) a_{n+1})
    cplx<T> bu1 = mk<T>(0, 0), bu2 = mk<T>(0, 0), bv1 = mk<T>(0, 0), bv2 = mk<T>(0, 0);
    cplx<T> ua = mk<T>(0, 0), va = mk<T>(0, 0);  // a_{n+1}
    for (int n = N - 1; n >= 0; --n) {
      const T two = (T)(2 * (n + 1));
      cplx<T> du = (n + 1 < N) ? bu2 + scl(ua, two) : mk<T>(0, 0);
      cplx<T> dv = (n + 1 < N) ? bv2 + scl(va, two) : mk<T>(0, 0);
      bu2 = bu1; bu1 = du;
      bv2 = bv1; bv1 = dv;
      if (n == 0) { du = scl(du, (T)0.5); dv = scl(dv, (T)0.5); }
      const cplx<T> u = ws.co(0, n), v = ws.co(1, n), w = ws.co(2, n);
      ws.co(3, n) = scl(mul_i(w), hky) - scl(dv, hs);
      ws.co(4, n) = scl(du, hs) - scl(mul_i(w), hkx);
      ws.co(5, n) = scl(mul_i(v), hkx) - scl(mul_i(u), hky);
      ua = u;
      va = v;
    }
  }

  // ---------------- F. inverse DCT-I to the occupied planes, 1/(Nx Ny) ----------------------------
  {
    const T scale = (T)(1.0 / ((double)g.nx * (double)g.ny));
    for (int o = 0; o < nfo; ++o) {
      for (int c0 = clo; c0 <= chi; c0 += NCH) {
        cplx<T> acc[NCH];
#pragma unroll
        for (int j = 0; j < NCH; ++j) acc[j] = mk<T>((T)0, (T)0);
        for (int n = 0; n < N; ++n) {
          const cplx<T> y = ws.co(o, n);
#pragma unroll
          for (int j = 0; j < NCH; ++j) {
            const int c = c0 + j;
            if (c <= chi) {
              const T im = ld<T>(tb.idct, c * N + n);
              acc[j].x += im * y.x;
              acc[j].y += im * y.y;
            }
          }
        }
#pragma unroll
        for (int j = 0; j < NCH; ++j)
          if (c0 + j <= chi) grid[gaddr(o, c0 + j)] = scl(acc[j], scale);
      }
    }
  }
}

template <typename T, int NCH>
__global__ void __launch_bounds__(kBvpThreads) bvp_kernel(Geometry g, BvpTabs tb, cplx<T>* __restrict__ grid,
                                                          const int* __restrict__ zrange, Ws<T> ws0) {
  const int clo = zrange[0], chi = zrange[1];
  const int64_t K = (int64_t)g.nkx * g.ny;
  Ws<T> ws = ws0;
  ws.slots = gridDim.x * blockDim.x;
  ws.slot = blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t k = ws.slot; k < K; k += ws.slots) solve_one<T, NCH>(g, tb, grid, clo, chi, k, ws);
}

template <typename T> constexpr int nch() { return sizeof(T) == 4 ? 33 : 17; }

}  // namespace

template <typename T>
size_t bvp_slot_bytes(const Plan& p) {
  const size_t N = (size_t)p.g.nz;
  return 7 * N * sizeof(cplx<T>) + 3 * N * sizeof(cplx<double>) + 3 * N * sizeof(double);
}

template <typename T>
int bvp_occupancy_blocks(const Plan& p) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bvp_kernel<T, nch<T>()>, kBvpThreads, 0);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 4) per_sm = 4;
  return per_sm * sms;
}

template <typename T>
void launch_bvp(const Plan& p, cudaStream_t s) {
  BvpTabs tb{p.tab.band, p.tab.dct, p.tab.dctd, p.tab.idct, p.tab.zeta};
  Ws<T> ws;
  const size_t N = (size_t)p.g.nz;
  const size_t slots = (size_t)p.bvp_blocks * kBvpThreads;
  unsigned char* base = reinterpret_cast<unsigned char*>(p.ws);
  ws.wt = reinterpret_cast<cplx<T>*>(base);
  ws.wd = reinterpret_cast<cplx<double>*>(base + 7 * N * slots * sizeof(cplx<T>));
  ws.wr = reinterpret_cast<double*>(base + 7 * N * slots * sizeof(cplx<T>) + 3 * N * slots * sizeof(cplx<double>));
  ws.N = (int)N;
  ws.slots = (int)slots;
  ws.slot = 0;
  bvp_kernel<T, nch<T>()><<<p.bvp_blocks, kBvpThreads, 0, s>>>(p.g, tb, reinterpret_cast<cplx<T>*>(p.grid), p.zrange, ws);
}

template size_t bvp_slot_bytes<float>(const Plan&);
template size_t bvp_slot_bytes<double>(const Plan&);
template int bvp_occupancy_blocks<float>(const Plan&);
template int bvp_occupancy_blocks<double>(const Plan&);
template void launch_bvp<float>(const Plan&, cudaStream_t);
template void launch_bvp<double>(const Plan&, cudaStream_t);

}  // namespace dps
