// Mixed-precision smoothing: FP32 Gauss-Seidel sweeps on the correction, inside FP64 defect
// correction (the FP32 form of the fast-sweeping smoother).
//
// A state f (FP64, Grad form) is improved by solving L e = d for a correction e, where
// d = r - R(f) is the FP64 defect and L a frozen-coefficient linearization of the operator at
// f: bases, HLL weights, time steps and collision frequencies are those of f; face states are
// reconstructed from the corrections as the FP64 operator reconstructs them from the state
// (eq. moments-recon), with the limiter's weights frozen at f (the van Albada slope
// ((b^2+e)a + (a^2+e)b) / (a^2+b^2+2e) becomes w_a da + w_b db with w_a, w_b taken from the
// state's differences a, b), in the face bases the state reconstructs, then re-expanded into
// the cell basis; the wall flux, being linear in the face state, is kept as is; the collision
// is nu (P e - e) with P the projection onto the conserved moments (the linear response of the
// local Maxwellian), plus the linearized Shakhov heat-flux term.  The correction is swept in
// FP32 with exactly the cell order of the FP64 smoother (Algorithm 1 applied to L e = d), then
// added to f in FP64 and projected back to Grad form.  (A first-order L for a second-order
// limited operator lets some modes stop contracting: the iteration then stalls near 1e-6.)  Because the unknown is the correction, its FP32 rounding error is relative
// to e, which shrinks with the defect: the outer FP64 iteration converges to the FP64 fixed
// point R(f) = r.
#include "nrmg_device.cuh"

namespace nrmg {

// ------------------------------------------------------------------ shared-memory layout (FP32)
struct CLayout {
  size_t cst, VA, VB, ss, vsrc, vdst, cf, sc, ti32, vflag, iarr, tu16, total;
};

__host__ __device__ inline CLayout make_corr_layout(int M, int N, int NP) {
  const int NE = nmom_even(M);
  CLayout s;
  size_t o = 0;
  size_t vb = (size_t)8 * (8 + NP), va = (size_t)kNV * NP;
  if (va > vb) vb = va;
  s.cst = o;   o = al16(o + sizeof(float) * (8 + NP));
  s.VA = o;    o = al16(o + sizeof(float) * kNV * NP);
  s.VB = o;    o = al16(o + sizeof(float) * vb);
  s.ss = o;    o = al16(o + sizeof(float) * 9 * NP);
  s.vsrc = o;  o = al16(o + sizeof(float) * kNV * 4);
  s.vdst = o;  o = al16(o + sizeof(float) * kNV * 4);
  s.cf = o;    o = al16(o + sizeof(float) * kNV * 3 * (M + 1));
  s.sc = o;    o = al16(o + sizeof(float) * 64);
  s.ti32 = o;  o = al16(o + sizeof(int) * (3 * NE + N));
  s.vflag = o; o = al16(o + sizeof(int) * kNV * 3);
  s.iarr = o;  o = al16(o + sizeof(int) * 64);
  s.tu16 = o;  o = al16(o + sizeof(uint16_t) * (13 * N + NE));
  s.total = o;
  return s;
}

__device__ inline SmT<float> bind_corr(char *base, int M, int N, int NP) {
  CLayout L = make_corr_layout(M, N, NP);
  SmT<float> s;
  s.cst = (float *)(base + L.cst);
  s.VA = (float *)(base + L.VA);
  s.VB = (float *)(base + L.VB);
  s.vsrc = (float *)(base + L.vsrc);
  s.vdst = (float *)(base + L.vdst);
  s.cf = (float *)(base + L.cf);
  s.sc = (float *)(base + L.sc);
  s.fact = nullptr;
  s.tslot = (int *)(base + L.ti32);
  s.tshak = s.tslot + 3 * nmom_even(M);
  s.vflag = (int *)(base + L.vflag);
  s.iarr = (int *)(base + L.iarr);
  s.tmem = (uint16_t *)(base + L.tu16);
  s.tprev = s.tmem + 3 * N;
  s.tnext = s.tmem + 6 * N;
  s.tal = s.tmem + 9 * N;
  s.tdeg = s.tmem + 12 * N;
  s.eidx = s.tmem + 13 * N;
  return s;
}

// correction stencil slots: 0 C, 1 E, 2 W, 3 N, 4 S, 5 EE, 6 WW, 7 NN, 8 SS; a row is
// [aux(8) | e(NP)]; the FP32 state of the same cells (limiter weights) sits in its own region
__device__ inline float *cstencil(const SmT<float> &s, int sl, int NP) {
  return sl == 0 ? s.cst : s.VB + (size_t)(sl - 1) * (8 + NP);
}
__device__ inline float *corr_state(char *base, int M, int N, int NP) {
  return (float *)(base + make_corr_layout(M, N, NP).ss);
}

// half of the limited slope of the frozen face bases (FP32 twin of the FP64 reconstruction)
__device__ inline float half_slope_f(int slope, float qm, float q0, float qp) {
  if (slope == 1) return 0.25f * (qp - qm);
  float a = q0 - qm, b = qp - q0;
  // the linearized operator only needs the weights approximately: fast division
  return __fdividef(0.5f * ((a + b) * fmaf(a, b, 1e-12f)), fmaf(a, a, fmaf(b, b, 2e-12f)));
}

enum { C_DT = 0, C_NU = 1, C_Q = 2 /* ..5 */, C_W = 8 /* ..8+12 */, C_RHOW = 20 /* ..24 */ };

// ------------------------------------------------------------------ frozen coefficients and FP32 defect
__global__ void mixed_prep_kernel(Consts K, LevelDev L) {
  const size_t tot = (size_t)L.ncell * K.NP;
  for (size_t q = (size_t)blockIdx.x * kThreads + threadIdx.x; q < tot; q += (size_t)gridDim.x * kThreads) {
    L.d32[q] = (float)L.D[q];
    L.e32[q] = 0.0f;
    L.s32[q] = (float)L.F[q];
  }
  for (int c = blockIdx.x * kThreads + threadIdx.x; c < L.ncell; c += gridDim.x * kThreads) {
    const double *p = L.P + (size_t)c * 4;
    const double rho = L.F[(size_t)c * K.NP], th = p[3], sq = sqrt(th);
    const double nu = K.nu0 * rho * L.tp[c];
    double dt = K.cfl / ((fabs(p[0]) + K.C * sq) * inv_hx(L, c % L.nx) + (fabs(p[1]) + K.C * sq) * inv_hy(L, c / L.nx));
    if (K.dtnu > 0.0) dt = fmin(dt, K.dtnu / nu);
    float *a = L.aux32 + (size_t)c * 8;
    for (int e = 0; e < 4; ++e) a[e] = (float)p[e];
    a[4] = (float)dt;
    a[5] = (float)nu;
    a[6] = 0.0f;
    a[7] = 0.0f;
  }
}

// ------------------------------------------------------------------ FP32 correction sweeps
__global__ void __launch_bounds__(kThreads) fs_corr_kernel(Consts K, LevelDev L, int steps, const int *queue) {
  extern __shared__ __align__(16) char smem_raw[];
  SmT<float> s = bind_corr(smem_raw, K.M, K.N, K.NP);
  float *ss = corr_state(smem_raw, K.M, K.N, K.NP);
  const int tid = threadIdx.x, N = K.N, NP = K.NP, NE = K.NE, M = K.M;
  for (int e = tid; e < 3 * NE + N; e += kThreads) s.tslot[e] = K.tab_i32[e];
  for (int e = tid; e < 13 * N + NE; e += kThreads) s.tmem[e] = K.tab_u16[e];
  __syncthreads();
  const int ncell = L.ncell;
  const long long total = (long long)steps * 4 * ncell;
  const float Cf = (float)K.C;
  for (;;) {
    if (tid == 0) {
      int it = atomicAdd(K.queue, 1);
      if (ld_volatile(K.abort_flag)) it = (int)total;
      s.iarr[I_ITEM] = it;
      s.iarr[I_ABW] = 0;
    }
    __syncthreads();
    const long long item = s.iarr[I_ITEM];
    if (item >= total) break;
    int st, k, c;
    if (queue) {
      const int qv = queue[item];
      st = qv / (4 * ncell);
      k = (qv / ncell) % 4;
      c = qv % ncell;
    } else {
      st = (int)(item / (4LL * ncell));
      k = (int)((item / ncell) % 4);
      c = L.order[(size_t)k * ncell + (int)(item % ncell)];
    }
    const int i = c % L.nx, j = c / L.nx;
    const int v = 4 * st + k + 1;
    // ---- per stencil slot (warp w takes slot w, warp 0 also slot 8): lane 0 waits until the
    //      cell holds the version of the serial order (the newest for a neighbour that sweep Dk
    //      visits earlier, the previous one otherwise), then the warp loads the cell's row:
    //      frozen coefficients, correction and FP32 state (even alpha_3 entries, kU loads in
    //      flight per lane).  A satisfied cell cannot change again before this update is
    //      published, so rows that are ready early load while the last dependency is pending.
    {
      const int warp = tid >> 5, lane = tid & 31;
      const int si = (k == 0 || k == 3) ? 1 : -1, sj = (k == 0 || k == 1) ? 1 : -1;
      for (int sl = warp; sl < 9; sl += kThreads / 32) {
        const int di = c_nb_di[sl], dj = c_nb_dj[sl];
        const int ii = i + di, jj = j + dj;
        const bool in = ii >= 0 && ii < L.nx && jj >= 0 && jj < L.ny && abs(di) + abs(dj) <= K.reach;
        int ok = 0;
        if (lane == 0) {
          s.iarr[I_EX + sl] = in ? 1 : 0;
          if (sl >= 1 && sl <= 4) s.iarr[I_WALL + sl - 1] = in ? 0 : 1;  // face f = slot f + 1
          if (in) {
            const bool before = (si * di < 0) || (di == 0 && sj * dj < 0);
            const int need = (sl != 0 && before) ? v : v - 1;
            const int *flag = L.ver + (size_t)jj * L.nx + ii;
            ok = 1;
            if (ld_acquire(flag) < need) {
              unsigned long long t0 = gtimer();
              while (ld_acquire(flag) < need) {
                if (ld_volatile(K.abort_flag)) {
                  ok = 0;
                  break;
                }
                if (gtimer() - t0 > kWaitLimitNs) {
                  raise_status(K, kStTimeout, true);
                  ok = 0;
                  break;
                }
                __nanosleep(32);
              }
            }
            if (!ok) s.iarr[I_ABW] = 1;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (ok) {
          const int cc = c + dj * L.nx + di;
          float *row = cstencil(s, sl, NP), *srow = ss + sl * NP;
          const int W = 8 + 2 * NE;
          constexpr int kU = 8;
          for (int q0 = lane; q0 < W; q0 += kU * 32) {
            float vv[kU];
            float *dd[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
              const int e = q0 + u * 32;
              dd[u] = nullptr;
              if (e < 8) {
                vv[u] = __ldcg(L.aux32 + (size_t)cc * 8 + e);
                dd[u] = row + e;
              } else if (e < 8 + NE) {
                const int o = s.eidx[e - 8];
                vv[u] = __ldcg(L.e32 + (size_t)cc * NP + o);
                dd[u] = row + 8 + o;
              } else if (e < W) {
                const int o = s.eidx[e - 8 - NE];
                vv[u] = L.s32[(size_t)cc * NP + o];  // written before the launch
                dd[u] = srow + o;
              }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u)
              if (dd[u]) *dd[u] = vv[u];
          }
        }
      }
    }
    __syncthreads();
    if (s.iarr[I_ABW]) break;
    const float *ac = s.cst, *ec = s.cst + 8;  // own frozen coefficients, own correction
    // ---- face states of the correction, slots as in the FP64 operator: 2f / 2f+1 = face f's
    //      left / right state (E, W, N, S), or 2f = the cell in the wall basis at a wall
    {
      const bool slopes = K.reach == 2 && K.slope != 0;
      const int tot = 6 * (4 + NE);
      for (int q = tid; q < tot; q += kThreads) {
        int it = q / (4 + NE), e = q - it * (4 + NE);
        int X = c_it_x[it], Xm = c_it_m[it], Xp = c_it_p[it];
        if (!s.iarr[I_EX + X]) continue;
        bool on = slopes && s.iarr[I_EX + Xm] && s.iarr[I_EX + Xp];
        const float *rx = cstencil(s, X, NP);
        // reconstruction factors of the item's cell: 1, 1, 1/4 on a uniform grid
        float rm = 1.0f, rp = 1.0f, ch = 0.25f;
        if (on && !L.uniform) {
          if (it == 1 || it >= 4) {
            const int r = j + c_nb_dj[X];
            rm = (float)L.rmy[r], rp = (float)L.rpy[r], ch = (float)L.chy[r];
          } else {
            const int col = i + c_nb_di[X];
            rm = (float)L.rmx[col], rp = (float)L.rpx[col], ch = (float)L.chx[col];
          }
        }
        float q0, hs = 0.0f;
        if (e < 4) {  // face basis: the reconstructed params of the state
          q0 = rx[e];
          if (on) {
            const float qm = cstencil(s, Xm, NP)[e], qp = cstencil(s, Xp, NP)[e];
            hs = L.uniform ? half_slope_f(K.slope, qm, q0, qp)
                           : (K.slope == 1 ? (qp - qm) * ch : half_slope_f(K.slope, q0 - (q0 - qm) * rm, q0, q0 + (qp - q0) * rp));
          }
        } else {      // correction: the limited slope linearized with frozen weights
          e = 4 + s.eidx[e - 4];
          const int o = e - 4;
          q0 = rx[8 + o];
          if (on) {
            const float em = cstencil(s, Xm, NP)[8 + o], ep = cstencil(s, Xp, NP)[8 + o];
            if (K.slope == 1) {
              hs = L.uniform ? 0.25f * (ep - em) : (ep - em) * ch;
            } else if (L.uniform) {
              const float a = ss[X * NP + o] - ss[Xm * NP + o], b = ss[Xp * NP + o] - ss[X * NP + o];
              const float den = fmaf(a, a, fmaf(b, b, 2e-12f));
              hs = __fdividef(0.5f * (fmaf(b, b, 1e-12f) * (q0 - em) + fmaf(a, a, 1e-12f) * (ep - q0)), den);
            } else {
              const float a = (ss[X * NP + o] - ss[Xm * NP + o]) * rm, b = (ss[Xp * NP + o] - ss[X * NP + o]) * rp;
              const float den = fmaf(a, a, fmaf(b, b, 2e-12f));
              hs = __fdividef(0.5f * (fmaf(b, b, 1e-12f) * (q0 - em) * rm + fmaf(a, a, 1e-12f) * (ep - q0) * rp), den);
            }
          }
        }
        int v0, v1 = -1;
        float x0, x1 = 0.0f;
        switch (it) {
          case 0:
            v0 = 0; x0 = q0 + hs;
            if (s.iarr[I_WALL + 1]) { v1 = 2; x1 = q0; } else { v1 = 3; x1 = q0 - hs; }
            break;
          case 1:
            v0 = 4; x0 = q0 + hs;
            if (s.iarr[I_WALL + 3]) { v1 = 6; x1 = q0; } else { v1 = 7; x1 = q0 - hs; }
            break;
          case 2: v0 = 1; x0 = q0 - hs; break;
          case 3: v0 = 2; x0 = q0 + hs; break;
          case 4: v0 = 5; x0 = q0 - hs; break;
          default: v0 = 6; x0 = q0 + hs; break;
        }
        if (e < 4) {
          s.vsrc[v0 * 4 + e] = x0;
          if (v1 >= 0) s.vsrc[v1 * 4 + e] = x1;
        } else {
          s.VA[v0 * NP + e - 4] = x0;
          if (v1 >= 0) s.VA[v1 * NP + e - 4] = x1;
        }
      }
    }
    // destination bases: the cell, or the wall for a wall face's slot 2f
    if (tid < 32) {
      int vv = tid >> 2, e = tid & 3, f = vv >> 1;
      if (s.iarr[I_WALL + f] && !(vv & 1)) {
        int w = c_face_wall[f];
        s.vdst[vv * 4 + e] = e < 3 ? (float)K.wall_u[w][e] : (float)K.wall_theta[w];
      } else {
        s.vdst[vv * 4 + e] = ac[e];
      }
    }
    if (tid == 32) {
      int na = 0;
      for (int f = 0; f < 4; ++f) {
        s.iarr[I_ACT + na++] = 2 * f;
        if (!s.iarr[I_WALL + f]) s.iarr[I_ACT + na++] = 2 * f + 1;
      }
      s.iarr[I_NACT] = na;
    }
    if (tid >= 96 && tid < 99 && K.model == 1) {
      int ii = tid - 96;
      const int *iq = K.tab_i32 + K.iq_off + 4 * ii;
      float qv = 2.0f * ec[iq[0]];
      for (int d = 0; d < 3; ++d) qv += ec[iq[1 + d]];
      s.sc[C_Q + ii] = (ii == 2) ? 0.0f : qv;  // q_3 involves only odd alpha_3 entries
    }
    __syncthreads();
    // frozen HLL weights of the reconstructed face bases
    if (tid >= 64 && tid < 68 && !s.iarr[I_WALL + tid - 64]) {
      int f = tid - 64, ax = f >> 1;
      const float *pl = s.vsrc + (2 * f) * 4, *pr = s.vsrc + (2 * f + 1) * 4;
      float sL = fminf(pl[ax] - Cf * sqrtf(pl[3]), pr[ax] - Cf * sqrtf(pr[3]));
      float sR = fmaxf(pl[ax] + Cf * sqrtf(pl[3]), pr[ax] + Cf * sqrtf(pr[3]));
      float w1, w2, w3;
      if (sL >= 0.0f) {
        w1 = 1.0f; w2 = 0.0f; w3 = 0.0f;
      } else if (sR <= 0.0f) {
        w1 = 0.0f; w2 = 1.0f; w3 = 0.0f;
      } else {
        float inv = 1.0f / (sR - sL);
        w1 = sR * inv; w2 = -sL * inv; w3 = sL * sR * inv;
      }
      s.sc[C_W + 3 * f] = w1;
      s.sc[C_W + 3 * f + 1] = w2;
      s.sc[C_W + 3 * f + 2] = w3;
    }
    setup_coeffs(K, s);
    __syncthreads();
    transform_batch(K, s, s.VA, s.VB);
    // ---- wall fluxes (linear in the face state)
    if (tid < 4 && s.iarr[I_WALL + tid]) {
      int w = c_face_wall[tid], ax = c_wall_axis[w];
      const float *a = s.VB + (2 * tid) * NP;
      const float *wr = K.wallRf + w * (M + 1);
      float rw = 0.0f;
      for (int m = 0; m <= M; ++m) rw = fmaf(wr[m], a[K.idx_axis[ax][m]], rw);
      s.sc[C_RHOW + tid] = rw;
    }
    __syncthreads();
    {
      int nw = 0, wf[4];
      for (int f = 0; f < 4; ++f)
        if (s.iarr[I_WALL + f]) wf[nw++] = f;
      for (int q = tid; q < nw * NE; q += kThreads) {
        int kk = q / NE, r = q - kk * NE;
        int f = wf[kk], w = c_face_wall[f], ax = c_wall_axis[w];
        int pk = s.tslot[ax * NE + r];
        int o = pk & 2047, s0 = (pk >> 11) & 2047, p = pk >> 22;
        int b0 = s0 - p, deg = s.tdeg[o];
        int Lm = M - (deg - p);
        const float *a = s.VB + (2 * f) * NP;
        const float *Wm = K.wallWf + (size_t)w * (M + 1) * (M + 1) + p * (M + 1);
        const uint16_t *mem = s.tmem + ax * N;
        float g = 0.0f;
        for (int m = 0; m <= Lm; ++m) g = fmaf(a[mem[b0 + m]], Wm[m], g);
        if (deg == p) g = fmaf(s.sc[C_RHOW + f], K.wallInf[w * (M + 1) + p], g);
        s.VA[(2 * f) * NP + o] = g;
      }
      if (tid == 0) {
        for (int kk = 0; kk < nw; ++kk) s.iarr[I_ACT + kk] = 2 * wf[kk];
        s.iarr[I_NACT] = nw;
      }
      if (tid < 4 && s.iarr[I_WALL + tid]) {
        int w = c_face_wall[tid];
        for (int e = 0; e < 4; ++e) {
          s.vsrc[(2 * tid) * 4 + e] = e < 3 ? (float)K.wall_u[w][e] : (float)K.wall_theta[w];
          s.vdst[(2 * tid) * 4 + e] = ac[e];
        }
      }
      __syncthreads();
      if (nw > 0) {
        setup_coeffs(K, s);
        __syncthreads();
        transform_batch(K, s, s.VA, s.VB);
      }
    }
    // ---- flux differences: F_E - F_W = Xi_x d_x + e_x, F_N - F_S = Xi_y d_y + e_y
    float *dX = s.VA, *dY = s.VA + NP, *eX = s.VA + 2 * NP, *eY = s.VA + 3 * NP;
    for (int q = tid; q < NE; q += kThreads) {
      const int o = s.eidx[q];
      float d[2] = {0.0f, 0.0f}, ee[2] = {0.0f, 0.0f};
#pragma unroll
      for (int fc = 0; fc < 4; ++fc) {
        int ax = fc >> 1;
        float sg = (fc & 1) ? -1.0f : 1.0f;
        if (s.iarr[I_WALL + fc]) {
          ee[ax] = fmaf(sg, s.VB[(2 * fc) * NP + o], ee[ax]);
        } else {
          float am = s.VB[(2 * fc) * NP + o], ap = s.VB[(2 * fc + 1) * NP + o];
          float w1 = s.sc[C_W + 3 * fc], w2 = s.sc[C_W + 3 * fc + 1], w3 = s.sc[C_W + 3 * fc + 2];
          d[ax] = fmaf(sg, fmaf(w1, am, w2 * ap), d[ax]);
          ee[ax] = fmaf(sg * w3, ap - am, ee[ax]);
        }
      }
      dX[o] = d[0];
      dY[o] = d[1];
      eX[o] = ee[0];
      eY[o] = ee[1];
    }
    __syncthreads();
    // ---- L e - d and the Gauss-Seidel update e <- e + dt (L e - d)
    const float nu = ac[5], dt = ac[4];
    const float idx = (float)inv_hx(L, i), idy = (float)inv_hy(L, j), shk = (float)((1.0 - K.Pr) * 0.2);
    const float e2m = (ec[K.idx_2e[0]] + ec[K.idx_2e[1]] + ec[K.idx_2e[2]]) * (1.0f / 3.0f);
    // ES-BGK: the degree-2 part of f^E is (1 - 1/Pr) times the trace-free degree-2 part of f
    // exactly; its degree >= 4 part is quadratic in the stress and is left out of the response
    const float esk = (float)(1.0 - 1.0 / K.Pr);
    const int i12 = K.tab_i32[K.iq_off + 12 + 1];
    float *Eo = L.e32 + (size_t)c * NP;
    const float *Do = L.d32 + (size_t)c * NP;
    for (int q = tid; q < NE; q += kThreads) {
      const int o = s.eidx[q];
      float xi[2];
#pragma unroll
      for (int ax = 0; ax < 2; ++ax) {
        const float *dd = ax == 0 ? dX : dY;
        uint16_t pr = s.tprev[ax * N + o], nx = s.tnext[ax * N + o];
        float vv = ac[ax] * dd[o];
        if (pr != 0xFFFF) vv = fmaf(ac[3], dd[pr], vv);
        if (nx != 0xFFFF) vv = fmaf((float)(s.tal[ax * N + o] + 1), dd[nx], vv);
        xi[ax] = vv;
      }
      // linear response of the equilibrium: the conserved moments of e (and the Shakhov term)
      float pe = 0.0f;
      if (o == 0 || o == K.idx_e[0] || o == K.idx_e[1])
        pe = ec[o];
      else if (o == K.idx_2e[0] || o == K.idx_2e[1] || o == K.idx_2e[2])
        pe = K.model == 2 ? fmaf(esk, ec[o] - e2m, e2m) : e2m;
      else if (K.model == 2 && o == i12)
        pe = esk * ec[o];
      if (K.model == 1) {
        int t = s.tshak[o];
        if (t >= 0) pe = fmaf(shk, s.sc[C_Q + t], pe);
      }
      float R = fmaf(-(xi[0] + eX[o]), idx, fmaf(-(xi[1] + eY[o]), idy, nu * (pe - ec[o])));
      Eo[o] = fmaf(dt, R - Do[o], ec[o]);
    }
    __syncthreads();  // orders the correction's writes before the release store
    if (tid == 0) st_release(L.ver + c, v);
  }
}

// ------------------------------------------------------------------ f <- Grad(f + e) in FP64
__device__ inline Sm bind_smem_f64(char *base, int M, int N, int NP) {
  SLayout Lo = make_layout(M, N, NP);
  Sm s;
  s.cst = (double *)(base + Lo.cst);
  s.VA = (double *)(base + Lo.VA);
  s.VB = (double *)(base + Lo.VB);
  s.vsrc = (double *)(base + Lo.vsrc);
  s.vdst = (double *)(base + Lo.vdst);
  s.cf = (double *)(base + Lo.cf);
  s.sc = (double *)(base + Lo.sc);
  s.fact = (double *)(base + Lo.fact);
  s.tslot = (int *)(base + Lo.ti32);
  s.tshak = s.tslot + 3 * nmom_even(M);
  s.vflag = (int *)(base + Lo.vflag);
  s.iarr = (int *)(base + Lo.iarr);
  s.tmem = (uint16_t *)(base + Lo.tu16);
  s.tprev = s.tmem + 3 * N;
  s.tnext = s.tmem + 6 * N;
  s.tal = s.tmem + 9 * N;
  s.tdeg = s.tmem + 12 * N;
  s.eidx = s.tmem + 13 * N;
  return s;
}

// Back to Grad form after adding the correction (the same projection as the FP64 sweep's).
__device__ inline bool regrad_mixed(const Consts &K, Sm &s, const double *pc) {
  const int tid = threadIdx.x, NP = K.NP;
  if (tid == 0) {
    const double *g = s.VA;
    double rho = g[0], f2 = 0.0, fe2 = 0.0, fe[3];
    const double ir = 1.0 / rho;
    for (int d = 0; d < 3; ++d) {
      fe[d] = d < 2 ? g[K.idx_e[d]] : 0.0;
      f2 += g[K.idx_2e[d]];
      fe2 += fe[d] * fe[d];
    }
    double th = fma(fma(2.0, f2, -fe2 * ir), ir * (1.0 / 3.0), pc[3]);
    for (int e = 0; e < 4; ++e) {
      double pn = e < 3 ? fma(fe[e], ir, pc[e]) : th;
      s.sc[S_NEWP + e] = pn;
      s.vsrc[e] = pc[e];
      s.vdst[e] = pn;
    }
    s.iarr[I_ACT] = 0;
    s.iarr[I_NACT] = 1;
    s.iarr[I_BAD] = !(isfinite(rho) && isfinite(th) && rho > 0.0 && th > 0.0);
  }
  __syncthreads();
  if (tid == kThreads - 1) s.sc[S_TPN] = pow(s.sc[S_NEWP + 3], 1.0 - K.omega);
  setup_coeffs(K, s);
  __syncthreads();
  transform_batch(K, s, s.VA, s.VB);
  double *g = s.VB;
  if (tid == 0) {
    for (int d = 0; d < 2; ++d) g[K.idx_e[d]] = 0.0;
    double s3 = (g[K.idx_2e[0]] + g[K.idx_2e[1]] + g[K.idx_2e[2]]) * (1.0 / 3.0);
    for (int d = 0; d < 3; ++d) g[K.idx_2e[d]] -= s3;
  }
  __syncthreads();
  int bad = 0;
  for (int q = tid; q < K.NE; q += kThreads) bad |= !isfinite(g[s.eidx[q]]);
  bad = __syncthreads_or(bad);
  (void)NP;
  return !(bad || s.iarr[I_BAD]);
}

__global__ void __launch_bounds__(kThreads) mixed_update_kernel(Consts K, LevelDev L) {
  extern __shared__ __align__(16) char smem_raw[];
  Sm s = bind_smem_f64(smem_raw, K.M, K.N, K.NP);
  const int tid = threadIdx.x, N = K.N, NE = K.NE, NP = K.NP;
  for (int e = tid; e < 3 * NE + N; e += kThreads) s.tslot[e] = K.tab_i32[e];
  for (int e = tid; e < 13 * N + NE; e += kThreads) s.tmem[e] = K.tab_u16[e];
  __syncthreads();
  for (int c = blockIdx.x; c < L.ncell; c += gridDim.x) {
    for (int q = tid; q < NE; q += kThreads) {
      const int o = s.eidx[q];
      s.VA[o] = L.F[(size_t)c * NP + o] + (double)L.e32[(size_t)c * NP + o];
    }
    __syncthreads();
    double pc[4];
    for (int e = 0; e < 4; ++e) pc[e] = L.P[(size_t)c * 4 + e];
    bool ok = regrad_mixed(K, s, pc);
    for (int q = tid; q < NE; q += kThreads) {
      const int o = s.eidx[q];
      L.F[(size_t)c * NP + o] = s.VB[o];
    }
    if (tid < 4) L.P[(size_t)c * 4 + tid] = s.sc[S_NEWP + tid];
    if (tid == 4) L.tp[c] = s.sc[S_TPN];
    if (!ok && tid == 0) atomicCAS(K.status, 0, kStNonPhysical);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ launchers
static void init_attrs_mixed() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(fs_corr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  cudaFuncSetAttribute(mixed_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  done = true;
}

cudaError_t launch_mixed_prep(const Consts &K, const LevelDev &L, cudaStream_t st) {
  size_t tot = (size_t)L.ncell * K.NP;
  int g = (int)((tot + kThreads - 1) / kThreads);
  if (g > 4096) g = 4096;
  mixed_prep_kernel<<<g, kThreads, 0, st>>>(K, L);
  return cudaGetLastError();
}

cudaError_t launch_fs_corr(const Consts &K, const LevelDev &L, int steps, const int *queue, int grid,
                           cudaStream_t st) {
  init_attrs_mixed();
  size_t sm = make_corr_layout(K.M, K.N, K.NP).total;
  fs_corr_kernel<<<grid, kThreads, sm, st>>>(K, L, steps, queue);
  return cudaGetLastError();
}

cudaError_t launch_mixed_update(const Consts &K, const LevelDev &L, int grid, cudaStream_t st) {
  init_attrs_mixed();
  size_t sm = make_layout(K.M, K.N, K.NP).total;
  mixed_update_kernel<<<grid, kThreads, sm, st>>>(K, L);
  return cudaGetLastError();
}

int occupancy_corr(int M, int NP) {
  init_attrs_mixed();
  int N = (M + 1) * (M + 2) * (M + 3) / 6;
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fs_corr_kernel, kThreads, make_corr_layout(M, N, NP).total);
  return nb;
}

}  // namespace nrmg
