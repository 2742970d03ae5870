// Device code of the GB300 nonlinear-multigrid moment solver (Hu & Li, arXiv 2206.13164).
//
// One CTA of kThreads threads updates one cell at a time.  A cell update needs up to nine
// re-expansions of a Hermite coefficient vector into another basis (Sec. 2.3); they are done
// together as one batched transform in shared memory, three directional passes with one
// output coefficient per thread, outputs ordered by the length of their index line so that the
// 32 lanes of a warp run loops of equal length.  The path is FP64-ALU bound: a cell update
// is tens of thousands of DFMAs against a few KB of state traffic.
//
// The Gauss-Seidel sweeps of Algorithm 1 run in one persistent launch per FS^s call.  CTAs take
// (step, sweep, cell) items from a global counter in anti-diagonal order and wait, on per-cell
// update counters, until every cell of the cross stencil holds exactly the version the serial
// order of the paper would show it: the newest one for a neighbour that sweep Dk visits earlier,
// the previous one otherwise.  This reproduces the serial sweep exactly while letting
// consecutive sweeps and steps overlap.  Every wait has a time limit after which the kernel
// records NRMG_ERR_TIMEOUT and all CTAs leave.  On small levels, where the wavefront is shorter
// than the GPU is wide, each cell update is split over a cluster of two CTAs on two SMs
// (fs_cluster_kernel).  Non-uniform grids take per-column and per-row widths (LevelDev geometry
// arrays); uniform grids keep their arithmetic.
#include "nrmg_device.cuh"

#include <algorithm>

namespace nrmg {

size_t cell_smem_bytes(int M, int NP) {
  int N = (M + 1) * (M + 2) * (M + 3) / 6;
  return make_layout(M, N, NP).total;
}

// ------------------------------------------------------------------ the cell operator
// ES-BGK (eq. ES-f^E): B = Lambda - theta I = (1 - 1/Pr) sigma / rho with sigma_dd = 2 f_{2e_d},
// sigma_12 = f_{e1+e2}; a planar state has sigma_13 = sigma_23 = 0, so exp(s^T B s / 2) factors
// into exp(B_dd s_d^2 / 2) (d = 1..3) and exp(B_12 s_1 s_2).  Threads 96..99 tabulate the factors'
// Taylor coefficients.
__device__ inline void es_factors(const int *is, double Pr, int M, const double *f, double *sc) {
  const int tid = threadIdx.x;
  if (tid < 96 || tid >= 100) return;
  const double kb = (1.0 - 1.0 / Pr) / f[0];
  if (tid < 99) {
    const int d = tid - 96;
    const double half_b = kb * f[is[d == 0 ? 0 : (d == 1 ? 3 : 5)]];  // B_dd / 2
    double t = 1.0;
    for (int m = 0; 2 * m <= M; ++m) {
      sc[S_ESG + d * (kMaxM / 2 + 1) + m] = t;
      t *= half_b / (m + 1);
    }
  } else {
    const double b12 = kb * f[is[1]];
    double t = 1.0;
    for (int k = 0; k <= M; ++k) {
      sc[S_ESH + k] = t;
      t *= b12 / (k + 1);
    }
  }
}

// f^E_alpha = rho [s^alpha] exp(s^T B s / 2) = rho g3(a3) sum_k B_12^k/k! g1(a1 - k) g2(a2 - k),
// gd(n) = (B_dd/2)^(n/2) / (n/2)! for even n and 0 for odd n; written to out[o] for every
// moment with even alpha_3 (eidx); tal holds alpha_1, alpha_2, alpha_3 of each moment.
__device__ inline void es_equilibrium(int N, int NE, const uint16_t *eidx, const uint16_t *tal,
                                            const double *sc, double rho, double *out) {
  const double *g = sc + S_ESG, *h = sc + S_ESH;
  for (int q = threadIdx.x; q < NE; q += kThreads) {
    const int o = eidx[q];
    const int a1 = tal[o], a2 = tal[N + o], a3 = tal[2 * N + o];
    double acc = 0.0;
    if (!((a1 ^ a2) & 1))
      for (int k = a1 & 1; k <= min(a1, a2); k += 2)
        acc = fma(h[k] * g[(a1 - k) >> 1], g[(kMaxM / 2 + 1) + ((a2 - k) >> 1)], acc);
    out[o] = rho * acc * g[2 * (kMaxM / 2 + 1) + (a3 >> 1)];
  }
}

// Loads the stencil of cell c (i,j) and computes, per coefficient, R_ij(f) - r_ij
// (eq. ode-system in the cell basis).  Threads receive elements o = tid, tid + kThreads, ...
// through emit(o, R_o - r_o).  kCoherent selects L2-only loads (the sweep kernel reads cells
// other CTAs have just written).  Transform vector slots: 2f / 2f+1 = face f's left / right
// state (E, W, N, S), or 2f = the cell re-expanded in the wall basis when face f is a wall;
// slot 8 = r.
// kES: the ES-BGK instantiation (model 2); the other models' instantiation carries no ES code.
// kPart: 0 the whole residual; 1 only the x faces (E, W), emitting -(F_E - F_W)/dx; 2 the y
// faces (N, S), the collision and r, emitting -(F_N - F_S)/dy + Q - r (the two halves of one
// cell update that a cluster of two CTAs computes side by side).
__host__ __device__ constexpr bool part_has_face(int part, int f) { return part == 0 || (part == 1) == (f < 2); }
// slope items of a part: 0 C along x, 1 C along y, 2 E, 3 W, 4 N, 5 S
__host__ __device__ constexpr int part_items(int part) { return part == 0 ? 6 : 3; }
__host__ __device__ constexpr int part_item(int part, int k) {
  return part == 0 ? k : (part == 1 ? (k == 0 ? 0 : k + 1) : (k == 0 ? 1 : k + 3));
}

template <bool kCoherent, bool kPreloaded = false, bool kES = false, int kPart = 0, typename Emit>
__device__ inline void cell_residual(const Consts &K, const LevelDev &L, Sm &s, int i, int j, Emit emit) {
  const int N = K.N, NP = K.NP, tid = threadIdx.x;
  const int c = j * L.nx + i;
  if (!kPreloaded && tid < 9) {
    int ii = i + c_nb_di[tid], jj = j + c_nb_dj[tid];
    int reach = abs(c_nb_di[tid]) + abs(c_nb_dj[tid]);
    s.iarr[I_EX + tid] = (ii >= 0 && ii < L.nx && jj >= 0 && jj < L.ny && reach <= K.reach) ? 1 : 0;
  }
  if (!kPreloaded) __syncthreads();
  // ---- stencil (params + the even-alpha_3 coefficients): each thread issues its loads
  //      before its shared-memory stores so that they are in flight together (kPreloaded:
  //      the caller has loaded the stencil and set the existence and wall flags)
  if (!kPreloaded) {
    const int NE = K.NE, W = 4 + NE, tot = 9 * W;
    constexpr int kU = 8;
    for (int q0 = tid; q0 < tot; q0 += kU * kThreads) {
      double v[kU];
      double *d[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        int q = q0 + u * kThreads;
        d[u] = nullptr;
        if (q < tot) {
          int sl = q / W, e = q - sl * W;
          if (s.iarr[I_EX + sl]) {
            int cc = c + c_nb_dj[sl] * L.nx + c_nb_di[sl];
            int col = e < 4 ? e : 4 + s.eidx[e - 4];
            const double *ptr = e < 4 ? L.P + (size_t)cc * 4 + e : L.F + (size_t)cc * NP + (col - 4);
            v[u] = kCoherent ? __ldcg(ptr) : *ptr;
            d[u] = stencil(s, sl, NP) + col;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (d[u]) *d[u] = v[u];
    }
  }
  if (!kPreloaded && tid < 4) s.iarr[I_WALL + tid] = s.iarr[I_EX + c_face_nb[tid]] ? 0 : 1;
  if (L.has_r && kPart != 1) {
    for (int e = tid; e < 4 + K.NE; e += kThreads) {
      if (e < 4) {
        s.vsrc[8 * 4 + e] = L.rP[(size_t)c * 4 + e];
      } else {
        const int o = s.eidx[e - 4];
        s.VA[8 * NP + o] = L.rF[(size_t)c * NP + o];
      }
    }
  }
  __syncthreads();
  const double *pc = s.cst;  // cell params, coefficients at pc + 4
  // ---- face states (eq. moments-recon): six slope items, each element computed once
  //   item 0: C along x -> slot 0 (E left) and slot 3 (W right), or slot 2 (W wall)
  //   item 1: C along y -> slot 4 (N left) and slot 7 (S right), or slot 6 (S wall)
  //   items 2..5: E -> slot 1, W -> slot 2, N -> slot 5, S -> slot 6
  const int NE = K.NE;
  // one slope item element: writes the face state(s) it feeds
  // one slope item element (item kk of the part, column e of the stencil rows: 0..3 the
  // params, 4 + o coefficient o): writes the face state(s) it feeds
  auto face_item = [&](int kk, int e) {
    const int it = part_item(kPart, kk);
    int X = c_it_x[it], Xm = c_it_m[it], Xp = c_it_p[it];
    if (!s.iarr[I_EX + X]) return;
    bool on = K.reach == 2 && K.slope != 0 && s.iarr[I_EX + Xm] && s.iarr[I_EX + Xp];
    double q0 = stencil(s, X, NP)[e];
    double hs = 0.0;
    if (on) {
      const double qm = stencil(s, Xm, NP)[e], qp = stencil(s, Xp, NP)[e];
      if (L.uniform) {
        hs = half_slope(K.slope, qm, q0, qp);
      } else if (it == 1 || it >= 4) {  // along y: the row of the item's cell
        const int r = j + c_nb_dj[X];
        hs = half_slope_nu(K.slope, qm, q0, qp, L.rmy[r], L.rpy[r], L.chy[r]);
      } else {
        const int col = i + c_nb_di[X];
        hs = half_slope_nu(K.slope, qm, q0, qp, L.rmx[col], L.rpx[col], L.chx[col]);
      }
    }
    int v0, v1 = -1;
    double x0, x1 = 0.0;
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
  };
  // The coefficient elements of the face states (the FP64-heavy part) run on every warp but the
  // last; the last warp meanwhile runs the short dependent chains that the transforms wait for:
  // the face states' basis params, the destination bases, the time step and collision
  // frequency, the HLL weights and the coefficients of the transform series.
  constexpr int kCoefThreads = kThreads - 32;
  if (tid < kCoefThreads) {
    const int tot = part_items(kPart) * NE;
    for (int q = tid; q < tot; q += 2 * kCoefThreads) {
      const int k0 = q / NE;
      face_item(k0, 4 + s.eidx[q - k0 * NE]);
      const int q1 = q + kCoefThreads;
      if (q1 < tot) {
        const int k1 = q1 / NE;
        face_item(k1, 4 + s.eidx[q1 - k1 * NE]);
      }
    }
    if (!kCoherent && tid == 64) {  // theta^-k of the norm weights (the residual kernel's norm)
      double it = 1.0 / pc[3], t = 1.0;
      for (int k = 0; k <= K.M; ++k) {
        s.sc[S_TPOW + k] = t;
        t *= it;
      }
    }
    if (tid >= 96 && tid < 99 && K.model == 1) {
      // q_i = 2 f_{3e_i} + sum_d f_{2e_d + e_i} (eq. moments-relation)
      int ii = tid - 96;
      const double *f = pc + 4;
      const int *iq = K.tab_i32 + K.iq_off + 4 * ii;
      double q = 2.0 * f[iq[0]];
      for (int d = 0; d < 3; ++d) q += f[iq[1 + d]];
      s.sc[S_Q + ii] = q;
    }
    if (kES) es_factors(K.tab_i32 + K.iq_off + 12, K.Pr, K.M, pc + 4, s.sc);
  } else {
    const int lane = tid - kCoefThreads;
    if (lane < part_items(kPart) * 4) face_item(lane >> 2, lane & 3);
    // destination bases: the cell, or the wall for a wall face's slot 2f
    for (int t = lane; t < 4 * kNV; t += 32) {
      int v = t >> 2, e = t & 3;
      int f = v >> 1;
      if (v < 8 && s.iarr[I_WALL + f] && !(v & 1)) {
        int w = c_face_wall[f];
        s.vdst[v * 4 + e] = e < 3 ? K.wall_u[w][e] : K.wall_theta[w];
      } else {
        s.vdst[v * 4 + e] = pc[e];
      }
    }
    if (lane == 0) {
      int na = 0;
      for (int f = 0; f < 4; ++f) {
        if (!part_has_face(kPart, f)) continue;
        s.iarr[I_ACT + na++] = 2 * f;
        if (!s.iarr[I_WALL + f]) s.iarr[I_ACT + na++] = 2 * f + 1;
      }
      if (L.has_r && kPart != 1) s.iarr[I_ACT + na++] = 8;
      s.iarr[I_NACT] = na;
    }
    __syncwarp();
    // lanes 0..3: HLL weights of interior face `lane`, F = w1 Xi a- + w2 Xi a+ + w3 (a+ - a-);
    // lane 4: the local time step (eq. local-CFL) and the collision frequency.  One code path:
    // two square roots, one reciprocal.
    if (lane < 5) {
      const int f = lane & 3, ax = f >> 1;
      const bool hll = lane < 4;
      const double *pm = hll ? s.vsrc + (2 * f) * 4 : pc, *pp = hll ? s.vsrc + (2 * f + 1) * 4 : pc;
      const double sm = sqrt(pm[3]), sp = sqrt(pp[3]);
      double sL = fmin(pm[ax] - K.C * sm, pp[ax] - K.C * sp);
      double sR = fmax(pm[ax] + K.C * sm, pp[ax] + K.C * sp);
      double den = sR - sL;
      if (!hll) den = (fabs(pc[0]) + K.C * sm) * inv_hx(L, i) + (fabs(pc[1]) + K.C * sm) * inv_hy(L, j);
      const double inv = 1.0 / den;
      if (hll) {
        if (!s.iarr[I_WALL + f] && part_has_face(kPart, f)) {
          double w1, w2, w3;
          if (sL >= 0.0) {
            w1 = 1.0; w2 = 0.0; w3 = 0.0;
          } else if (sR <= 0.0) {
            w1 = 0.0; w2 = 1.0; w3 = 0.0;
          } else {
            w1 = sR * inv; w2 = -sL * inv; w3 = sL * sR * inv;
          }
          s.sc[S_W + 3 * f] = w1;
          s.sc[S_W + 3 * f + 1] = w2;
          s.sc[S_W + 3 * f + 2] = w3;
        }
      } else {
        const double tpc = kCoherent ? __ldcg(L.tp + c) : L.tp[c];
        const double nu = K.nu0 * pc[4] * tpc;
        s.sc[S_NU] = nu;
        double dt = K.cfl * inv;
        if (K.dtnu > 0.0) dt = fmin(dt, K.dtnu / nu);
        s.sc[S_DT] = dt;
      }
    }
    __syncwarp();
    // series coefficients of every active vector and direction (setup_coeffs on this warp)
    {
      const int M = K.M, na = s.iarr[I_NACT];
      for (int t = lane; t < na * 3; t += 32) {
        int v = s.iarr[I_ACT + t / 3], d = t % 3;
        double a = s.vdst[v * 4 + d] - s.vsrc[v * 4 + d];
        double b = 0.5 * (s.vdst[v * 4 + 3] - s.vsrc[v * 4 + 3]);
        double *cf = s.cf + (v * 3 + d) * (M + 1);
        double cm = 1.0, ck = -a;
        cf[0] = cm;
        cf[1] = ck;
#pragma unroll
        for (int k = 1; k < kMaxM; ++k) {
          if (k >= M) break;
          double u = (-2.0 * b * cinv(0.0, k)) * cm;
          double cn = fma(-a * cinv(0.0, k), ck, u);
          cf[k + 1] = cn;
          cm = ck;
          ck = cn;
        }
        s.vflag[v * 3 + d] = ((a == 0.0 && b == 0.0) ? 1 : 0) | (a == 0.0 ? 2 : 0);
      }
    }
  }
  __syncthreads();
  // ---- batch A: face states -> cell basis, cell -> wall bases, r -> cell basis (result in VB)
  transform_batch(K, s, s.VA, s.VB);
  // ---- wall fluxes (half-range kinetic flux in the wall basis)
  if (tid < 4 && s.iarr[I_WALL + tid] && part_has_face(kPart, tid)) {
    int w = c_face_wall[tid], ax = c_wall_axis[w];
    const double *a = s.VB + (2 * tid) * NP;
    const double *wr = K.wallRho + w * (K.M + 1);
    double rw = 0.0;
    for (int m = 0; m <= K.M; ++m) rw += wr[m] * a[K.idx_axis[ax][m]];
    s.sc[S_RHOW + tid] = rw;
  }
  __syncthreads();
  {
    int nw = 0, wf[4];
    for (int f = 0; f < 4; ++f)
      if (s.iarr[I_WALL + f] && part_has_face(kPart, f)) wf[nw++] = f;
    for (int q = tid; q < nw * NE; q += kThreads) {
      int k = q / NE, r = q - k * NE;
      int f = wf[k], w = c_face_wall[f], ax = c_wall_axis[w];
      int pk = s.tslot[ax * NE + r];
      int o = pk & 2047, s0 = (pk >> 11) & 2047, p = pk >> 22;
      int b0 = s0 - p, deg = s.tdeg[o];
      int Lm = K.M - (deg - p);
      const double *a = s.VB + (2 * f) * NP;
      const double *W = K.wallW + (size_t)w * (K.M + 1) * (K.M + 1) + p * (K.M + 1);
      const uint16_t *mem = s.tmem + ax * N;
      double g = 0.0;
      for (int m = 0; m <= Lm; ++m) g = fma(a[mem[b0 + m]], W[m], g);
      if (deg == p) g = fma(s.sc[S_RHOW + f], K.wallIn[w * (K.M + 1) + p], g);
      s.VA[(2 * f) * NP + o] = g;
    }
    if (tid == 0) {
      int na = 0;
      for (int k = 0; k < nw; ++k) s.iarr[I_ACT + na++] = 2 * wf[k];
      s.iarr[I_NACT] = na;
    }
    if (tid < 4 && s.iarr[I_WALL + tid] && part_has_face(kPart, tid)) {
      int w = c_face_wall[tid];
      double *src = s.vsrc + (2 * tid) * 4, *dst = s.vdst + (2 * tid) * 4;
      for (int e = 0; e < 4; ++e) {
        src[e] = e < 3 ? K.wall_u[w][e] : K.wall_theta[w];
        dst[e] = pc[e];
      }
    }
    __syncthreads();
    if (nw > 0) {
      setup_coeffs(K, s);
      __syncthreads();
      // ---- batch B: wall fluxes back into the cell basis (VA -> VB, wall slots only)
      transform_batch(K, s, s.VA, s.VB);
    }
  }
  // ---- flux differences per axis: F_E - F_W = Xi_x d_x + e_x, F_N - F_S = Xi_y d_y + e_y
  //      with d = sum_f sign_f (w1 a- + w2 a+), e = sum_f sign_f w3 (a+ - a-) (+ wall fluxes)
  double *dX = s.VA, *dY = s.VA + NP, *eX = s.VA + 2 * NP, *eY = s.VA + 3 * NP;
  for (int q = tid; q < NE; q += kThreads) {
    const int o = s.eidx[q];
    double d[2] = {0.0, 0.0}, ee[2] = {0.0, 0.0};
#pragma unroll
    for (int fc = 0; fc < 4; ++fc) {
      if (!part_has_face(kPart, fc)) continue;
      int ax = fc >> 1;
      double sg = (fc & 1) ? -1.0 : 1.0;
      if (s.iarr[I_WALL + fc]) {
        ee[ax] = fma(sg, s.VB[(2 * fc) * NP + o], ee[ax]);
      } else {
        double am = s.VB[(2 * fc) * NP + o], ap = s.VB[(2 * fc + 1) * NP + o];
        double w1 = s.sc[S_W + 3 * fc], w2 = s.sc[S_W + 3 * fc + 1], w3 = s.sc[S_W + 3 * fc + 2];
        d[ax] = fma(sg, fma(w1, am, w2 * ap), d[ax]);
        ee[ax] = fma(sg * w3, ap - am, ee[ax]);
      }
    }
    dX[o] = d[0];
    dY[o] = d[1];
    eX[o] = ee[0];
    eY[o] = ee[1];
  }
  if (kES && kPart != 1) es_equilibrium(N, NE, s.eidx, s.tal, s.sc, pc[4], s.VA + 5 * NP);
  __syncthreads();
  // ---- R = -(F_E - F_W)/dx - (F_N - F_S)/dy + Q
  const double *f = pc + 4;
  const double nu = s.sc[S_NU];
  const double idx_c = inv_hx(L, i), idy_c = inv_hy(L, j);
  for (int q = tid; q < NE; q += kThreads) {
    const int o = s.eidx[q];
    double xi[2];
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
      if ((kPart == 1 && ax == 1) || (kPart == 2 && ax == 0)) {
        xi[ax] = 0.0;
        continue;
      }
      const double *dd = ax == 0 ? dX : dY;
      uint16_t pr = s.tprev[ax * N + o], nx = s.tnext[ax * N + o];
      double v = pc[ax] * dd[o];
      if (pr != kNone) v = fma(pc[3], dd[pr], v);
      if (nx != kNone) v = fma((double)(s.tal[ax * N + o] + 1), dd[nx], v);
      xi[ax] = v;
    }
    double fE = 0.0;
    if (o == 0) {
      fE = f[0];
    } else if (K.model == 1) {
      int t = s.tshak[o];
      if (t >= 0) fE = (1.0 - K.Pr) * s.sc[S_Q + t] * 0.2;
    } else if (kES) {
      fE = s.VA[5 * NP + o];
    }
    double Q = nu * (fE - f[o]);
    if (kPart == 1) {  // the x half: -(F_E - F_W)/dx only
      emit(o, -(xi[0] + eX[o]) * idx_c);
      continue;
    }
    double R = kPart == 0 ? fma(-(xi[0] + eX[o]), idx_c, fma(-(xi[1] + eY[o]), idy_c, Q))
                          : fma(-(xi[1] + eY[o]), idy_c, Q);
    double r = L.has_r ? s.VB[8 * NP + o] : 0.0;
    emit(o, R - r);
  }
}

// Back to Grad form (Sec. 2.4): macroscopics of g (basis pc), project g into the new basis,
// zero f_{e_d} and the round-off mean of f_{2e_d}.  g lives in VA slot `v`; the result is left
// in VB slot `v` and the new params in sc[S_NEWP..].  Returns true when the state is physical.
__device__ inline bool regrad(const Consts &K, Sm &s, const double *pc, int v, bool want_tp = false) {
  const int tid = threadIdx.x, NP = K.NP;
  if (tid == 0) {
    double mac[5];
    macros(K, pc, s.VA + v * NP, mac);
    for (int e = 0; e < 4; ++e) {
      s.sc[S_NEWP + e] = mac[1 + e];
      s.vsrc[v * 4 + e] = pc[e];
      s.vdst[v * 4 + e] = mac[1 + e];
    }
    s.iarr[I_ACT] = v;
    s.iarr[I_NACT] = 1;
    s.iarr[I_BAD] = !(isfinite(mac[0]) && isfinite(mac[4]) && mac[0] > 0.0 && mac[4] > 0.0);
  }
  __syncthreads();
  // theta^(1-omega) of the new state, on the last warp.  When the one-vector transform leaves
  // that warp without outputs (N_E <= kThreads - 32), the other warps synchronize among
  // themselves until the final barrier, so the power's latency overlaps the transform.
  const bool split = want_tp && K.NE <= kThreads - 32;
  const int nbar = split ? kThreads - 32 : kThreads;
  double *g = s.VB + v * NP;
  if (want_tp && tid == kThreads - 1) s.sc[S_TPN] = pow(s.sc[S_NEWP + 3], 1.0 - K.omega);
  if (!split || tid < kThreads - 32) {
    setup_coeffs(K, s);
    if (split)
      bar_first(nbar);
    else
      __syncthreads();
    transform_batch(K, s, s.VA, s.VB, nbar);
    if (tid == 0) {
      for (int d = 0; d < 2; ++d) g[K.idx_e[d]] = 0.0;  // f_{e_3} is not formed (odd alpha_3)
      double s3 = (g[K.idx_2e[0]] + g[K.idx_2e[1]] + g[K.idx_2e[2]]) * (1.0 / 3.0);
      for (int d = 0; d < 3; ++d) g[K.idx_2e[d]] -= s3;
    }
    if (split)
      bar_first(nbar);
    else
      __syncthreads();
  }
  int bad = 0;
  for (int q = tid; q < K.NE; q += kThreads) bad |= !isfinite(g[s.eidx[q]]);
  bad = __syncthreads_or(bad);
  return !(bad || s.iarr[I_BAD]);
}

// ------------------------------------------------------------------ FS^steps (Algorithm 1)
// One sweep item: update cell c (i,j) of sweep k to version v once the cross stencil holds
// the versions of the serial order (the newest for a neighbour that sweep Dk visits earlier,
// the previous one otherwise), then publish v.  Returns false when the launch must stop.
// stencil slots of a part: all nine, or the cell and its neighbours along x (E, W, EE, WW) or
// along y (N, S, NN, SS)
__host__ __device__ constexpr bool part_has_slot(int part, int sl) {
  return part == 0 || sl == 0 || (part == 1) == (sl == 1 || sl == 2 || sl == 5 || sl == 6);
}

// Dependency waits and stencil loads of one sweep item (the slots of part kPart; the existence
// and wall flags of all nine slots are set either way).  Returns after the CTA barrier; a wait
// that gave up sets iarr[I_ABW].
template <int kPart>
__device__ inline void fs_wait_load(const Consts &K, const LevelDev &L, Sm &s, int c, int k, int v) {
  const int tid = threadIdx.x, NP = K.NP, NE = K.NE;
  const int i = c % L.nx, j = c / L.nx;
  // ---- per stencil slot (warp w takes slot w, warp 0 also slot 8): lane 0 waits until the
  //      cell holds the version of the serial order (sweep Dk: i ascending for D1, D4; j
  //      ascending for D1, D2; outer loop i, inner j), then the warp loads the cell's params
  //      and even-alpha_3 coefficients (kU loads in flight per lane).  A satisfied cell cannot
  //      change again before this update is published, so rows that are ready early load
  //      while the last dependency is pending.
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
        if (in && part_has_slot(kPart, sl)) {
          const bool before = (si * di < 0) || (di == 0 && sj * dj < 0);
          const int need = (sl != 0 && before) ? v : v - 1;
          const int *flag = L.ver + (size_t)jj * L.nx + ii;
          ok = 1;
          if (ld_acquire(flag) < need) {
            // one load latency per round: the abort word (another global load) is read on
            // every 16th round only, the time limit on every round
            unsigned long long t0 = gtimer();
            for (int it = 1; ld_acquire(flag) < need; ++it) {
              if ((it & 15) == 0 && ld_volatile(K.abort_flag)) {
                ok = 0;
                break;
              }
              if (gtimer() - t0 > kWaitLimitNs) {
                raise_status(K, kStTimeout, true);
                ok = 0;
                break;
              }
            }
          }
          if (!ok) s.iarr[I_ABW] = 1;
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (ok) {
        const int cc = c + dj * L.nx + di;
        double *row = stencil(s, sl, NP);
        const int W = 4 + NE;
        constexpr int kU = 8;
        for (int q0 = lane; q0 < W; q0 += kU * 32) {
          double vv[kU];
          double *dd[kU];
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const int e = q0 + u * 32;
            dd[u] = nullptr;
            if (e < W) {
              const int col = e < 4 ? e : 4 + s.eidx[e - 4];
              const double *ptr = e < 4 ? L.P + (size_t)cc * 4 + e : L.F + (size_t)cc * NP + (col - 4);
              vv[u] = __ldcg(ptr);
              dd[u] = row + col;
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
}

template <bool kES>
__device__ inline bool fs_item(const Consts &K, const LevelDev &L, Sm &s, int c, int k, int v) {
  const int tid = threadIdx.x, NP = K.NP;
  const int i = c % L.nx, j = c / L.nx;
  fs_wait_load<0>(K, L, s, c, k, v);
  if (s.iarr[I_ABW]) return false;
  // ---- R_ij(f) - r_ij, then f + dt (R - r) into VA slot 4, back to Grad form
  cell_residual<true, true, kES>(K, L, s, i, j,
                            [&](int o, double Rr) { s.VA[4 * NP + o] = fma(s.sc[S_DT], Rr, s.cst[4 + o]); });
  __syncthreads();
  double pcell[4];
  for (int e = 0; e < 4; ++e) pcell[e] = s.cst[e];
  bool ok = regrad(K, s, pcell, 4, true);
  double *Fo = L.F + (size_t)c * NP;
  for (int q = tid; q < K.NE; q += kThreads) {
    const int o = s.eidx[q];
    Fo[o] = s.VB[4 * NP + o];
  }
  if (tid < 4) L.P[(size_t)c * 4 + tid] = s.sc[S_NEWP + tid];
  if (tid == 4) L.tp[c] = s.sc[S_TPN];
  if (!ok && tid == 0) raise_status(K, kStNonPhysical, true);
  // the barrier orders every thread's writes of the cell before thread 0's release store
  // (gpu scope), which the dependants' acquire loads synchronize with
  __syncthreads();
  if (tid == 0) st_release(L.ver + c, v);
  return true;
}

template <bool kES>
__global__ void __launch_bounds__(kThreads) fs_kernel(Consts K, LevelDev L, int steps, const int *queue) {
  extern __shared__ __align__(16) char smem_raw[];
  Sm s = bind_smem(smem_raw, K.M, K.N, K.NP);
  load_tables(K, s);
  __syncthreads();
  const int tid = threadIdx.x;
  const int ncell = L.ncell;
  const long long total = (long long)steps * 4 * ncell;
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
    if (!fs_item<kES>(K, L, s, c, k, 4 * st + k + 1)) break;
  }
}

// ------------------------------------------------------------------ FS^steps on a cluster of two CTAs
// On levels whose wavefront is shorter than the GPU is wide, one cell update is split over a
// cluster of two CTAs on two SMs (the FP64 pipe of one SM bounds a single update): CTA 0 takes
// the x faces (E, W: their face states, basis transforms, HLL or wall fluxes) and produces
// -(F_E - F_W)/dx; CTA 1 takes the y faces, r and the collision, adds CTA 0's half read from
// its shared memory (distributed shared memory of the cluster), updates the cell and projects
// it back to Grad form.  CTA 0 fetches the work items and hands each to CTA 1 through a mailbox
// in CTA 1's shared memory; with two exchange buffers it starts the next item while CTA 1
// finishes the current one.  Every wait on the partner is bounded like the dependency waits.
__device__ inline unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ inline unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// address of the same shared-memory location in CTA `rank` of the cluster
__device__ inline unsigned cluster_map(unsigned a, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ inline void st_cluster(unsigned a, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ inline void st_release_cluster(unsigned a, int v) {
  asm volatile("st.release.cluster.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ inline int ld_acquire_cluster(unsigned a) {
  int v;
  asm volatile("ld.acquire.cluster.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ inline double ld_cluster_f64(unsigned a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}
__device__ inline void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// bounded wait until the word at cluster address a holds at least `need`
__device__ inline bool wait_cluster_word(const Consts &K, unsigned a, int need) {
  if (ld_acquire_cluster(a) >= need) return true;
  const unsigned long long t0 = gtimer();
  while (ld_acquire_cluster(a) < need) {
    if (ld_volatile(K.abort_flag)) return false;
    if (gtimer() - t0 > kWaitLimitNs) {
      raise_status(K, kStTimeout, true);
      return false;
    }
    __nanosleep(32);
  }
  return true;
}

// exchange area behind the cell working set: x halves [2][NP] doubles, then control words
// (mailbox items [2], mailbox sequence, x-half sequence, consumed sequence)
enum { X_MBOX = 0, X_MSEQ = 2, X_FSEQ = 3, X_CSEQ = 4, X_WORDS = 8 };
__host__ __device__ inline size_t xchg_offset(int M, int N, int NP) { return al16(make_layout(M, N, NP).total); }
__host__ __device__ inline size_t cluster_smem_bytes(int M, int N, int NP) {
  return xchg_offset(M, N, NP) + sizeof(double) * 2 * NP + sizeof(int) * X_WORDS;
}
// at least this much dynamic shared memory per CTA: with one CTA per SM the two CTAs of a
// cluster never share an SM (and its FP64 pipe); with two per SM, two clusters share a pair
constexpr size_t kClusterMinSmem[2] = {120 * 1024, 78 * 1024};

// CTA 0 of a cluster: the x half of the update of cell c, written to this CTA's exchange
// buffer xh; then tells CTA 1 (x-half sequence n + 1 in its control words).
template <bool kES>
__device__ inline bool fs_item_x(const Consts &K, const LevelDev &L, Sm &s, int c, int k, int v, double *xh,
                                 unsigned peer_ctl, int n) {
  const int i = c % L.nx, j = c / L.nx;
  fs_wait_load<1>(K, L, s, c, k, v);
  if (s.iarr[I_ABW]) return false;
  cell_residual<true, true, kES, 1>(K, L, s, i, j, [&](int o, double Rx) { xh[o] = Rx; });
  // the barrier orders every thread's writes of xh before thread 0's release store (cluster
  // scope), which CTA 1's acquire load synchronizes with
  __syncthreads();
  if (threadIdx.x == 0) st_release_cluster(peer_ctl + 4 * X_FSEQ, n + 1);
  return true;
}

// CTA 1 of a cluster: the y half, r and the collision; then CTA 0's x half (read from its
// shared memory at cluster address peer_xh once the x-half sequence reaches n + 1), the update
// f + dt (R - r), the projection back to Grad form, the cell's write and its release.
template <bool kES>
__device__ inline bool fs_item_y(const Consts &K, const LevelDev &L, Sm &s, int c, int k, int v, unsigned peer_xh,
                                 unsigned my_ctl, unsigned peer_ctl, int n) {
  const int tid = threadIdx.x, NP = K.NP;
  const int i = c % L.nx, j = c / L.nx;
  fs_wait_load<2>(K, L, s, c, k, v);
  if (s.iarr[I_ABW]) return false;
  cell_residual<true, true, kES, 2>(K, L, s, i, j, [&](int o, double Ry) { s.VA[4 * NP + o] = Ry; });
  if (tid == 0 && !wait_cluster_word(K, my_ctl + 4 * X_FSEQ, n + 1)) s.iarr[I_ABW] = 1;
  __syncthreads();
  if (s.iarr[I_ABW]) return false;
  const double dt = s.sc[S_DT];
  for (int q = tid; q < K.NE; q += kThreads) {
    const int o = s.eidx[q];
    const double rx = ld_cluster_f64(peer_xh + 8u * (unsigned)o);
    s.VA[4 * NP + o] = fma(dt, rx + s.VA[4 * NP + o], s.cst[4 + o]);
  }
  __syncthreads();
  if (tid == 0) st_release_cluster(peer_ctl + 4 * X_CSEQ, n + 1);  // CTA 0 may reuse the buffer
  double pcell[4];
  for (int e = 0; e < 4; ++e) pcell[e] = s.cst[e];
  bool ok = regrad(K, s, pcell, 4, true);
  double *Fo = L.F + (size_t)c * NP;
  for (int q = tid; q < K.NE; q += kThreads) {
    const int o = s.eidx[q];
    Fo[o] = s.VB[4 * NP + o];
  }
  if (tid < 4) L.P[(size_t)c * 4 + tid] = s.sc[S_NEWP + tid];
  if (tid == 4) L.tp[c] = s.sc[S_TPN];
  if (!ok && tid == 0) raise_status(K, kStNonPhysical, true);
  __syncthreads();
  if (tid == 0) st_release(L.ver + c, v);
  return true;
}

template <bool kES>
__global__ void __launch_bounds__(kThreads) fs_cluster_kernel(Consts K, LevelDev L, int steps, const int *queue) {
  extern __shared__ __align__(16) char smem_raw[];
  Sm s = bind_smem(smem_raw, K.M, K.N, K.NP);
  load_tables(K, s);
  const int tid = threadIdx.x, NP = K.NP;
  const unsigned rank = cluster_rank(), peer = rank ^ 1u;
  double *xh = (double *)(smem_raw + xchg_offset(K.M, K.N, NP));
  int *ctl = (int *)(xh + 2 * NP);
  if (tid < X_WORDS) ctl[tid] = 0;
  __syncthreads();
  cluster_sync_all();  // both CTAs' control words are zero before either writes the other's
  const unsigned my_ctl = cluster_map(smem_addr(ctl), rank), peer_ctl = cluster_map(smem_addr(ctl), peer);
  const unsigned peer_xh0 = cluster_map(smem_addr(xh), peer);
  const int ncell = L.ncell;
  const long long total = (long long)steps * 4 * ncell;
  for (int n = 0;; ++n) {
    if (tid == 0) {
      int it = (int)total;
      if (rank == 0) {
        // the exchange buffer of item n was last used by item n - 2: CTA 1 must be done with it
        if ((n < 2 || wait_cluster_word(K, my_ctl + 4 * X_CSEQ, n - 1)) && !ld_volatile(K.abort_flag))
          it = atomicAdd(K.queue, 1);
        if (it > (int)total) it = (int)total;
        st_cluster(peer_ctl + 4 * (X_MBOX + (n & 1)), it);
        st_release_cluster(peer_ctl + 4 * X_MSEQ, n + 1);
      } else if (wait_cluster_word(K, my_ctl + 4 * X_MSEQ, n + 1)) {
        it = ctl[X_MBOX + (n & 1)];
      }
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
    const int v = 4 * st + k + 1;
    const bool ok = rank == 0 ? fs_item_x<kES>(K, L, s, c, k, v, xh + (n & 1) * NP, peer_ctl, n)
                              : fs_item_y<kES>(K, L, s, c, k, v, peer_xh0 + 8u * (unsigned)((n & 1) * NP), my_ctl,
                                               peer_ctl, n);
    if (!ok) {
      // leaving early: release the partner from its mailbox wait
      if (rank == 0 && tid == 0) {
        st_cluster(peer_ctl + 4 * (X_MBOX + ((n + 1) & 1)), (int)total);
        st_release_cluster(peer_ctl + 4 * X_MSEQ, n + 2);
      }
      break;
    }
  }
  __syncthreads();
  cluster_sync_all();  // neither CTA leaves while the other may still read its shared memory
}

// FS sweeps of several problems (same scheme, any M) in one persistent launch.  items[q] =
// (problem, item of that problem's level queue); the problem descriptors (scheme constants
// and level) are copied into shared memory per item.  K0 is the descriptor of the largest M:
// the dynamic shared memory is sized for it, and the working set of a smaller M fits in its
// layout; when the next item's M differs from the one whose index tables the CTA holds, the
// CTA rebinds its shared memory and loads that M's tables.  All descriptors share one abort
// word.
template <bool kES>
__global__ void __launch_bounds__(kThreads) fs_batch_kernel(const BatchDesc *desc, const int2 *items,
                                                            long long total, int *counter, Consts K0) {
  extern __shared__ __align__(16) char smem_raw[];
  __shared__ BatchDesc bd;
  Sm s = bind_smem(smem_raw, K0.M, K0.N, K0.NP);
  load_tables(K0, s);
  __syncthreads();
  const int tid = threadIdx.x;
  int cur = -1, curM = K0.M;
  for (;;) {
    if (tid == 0) {
      int it = atomicAdd(counter, 1);
      if (ld_volatile(K0.abort_flag)) it = (int)total;
      s.iarr[I_ITEM] = it;
      s.iarr[I_ABW] = 0;
    }
    __syncthreads();
    const long long item = s.iarr[I_ITEM];
    if (item >= total) break;
    const int2 iv = items[item];
    if (iv.x != cur) {  // uniform: every thread read the same item
      const int *src = (const int *)(desc + iv.x);
      int *dst = (int *)&bd;
      for (int w = tid; w < (int)(sizeof(BatchDesc) / sizeof(int)); w += kThreads) dst[w] = src[w];
      cur = iv.x;
      __syncthreads();
      if (bd.K.M != curM) {  // uniform: bd is shared; the item is already in a register
        s = bind_smem(smem_raw, bd.K.M, bd.K.N, bd.K.NP);
        load_tables(bd.K, s);
        curM = bd.K.M;
        if (tid == 0) s.iarr[I_ABW] = 0;  // the control words moved with the layout
        __syncthreads();
      }
    }
    const int ncell = bd.L.ncell, qv = iv.y;
    const int st = qv / (4 * ncell), k = (qv / ncell) % 4, c = qv % ncell;
    if (!fs_item<kES>(bd.K, bd.L, s, c, k, 4 * st + k + 1)) break;
  }
}

// ------------------------------------------------------------------ residual of every cell
// mode kResOut: out[c*stride + o] = R - r and the weighted norm partials;
// kResDefect: D = -(R - r); kResCoarseRhs: rF = R + rF (the level has no r during the call);
// kResDefectNorm: D = -(R - r) and the norm partials.
template <bool kES>
__global__ void __launch_bounds__(kThreads) residual_kernel(Consts K, LevelDev L, int mode, double *out,
                                                            int out_stride, double *partials) {
  extern __shared__ __align__(16) char smem_raw[];
  Sm s = bind_smem(smem_raw, K.M, K.N, K.NP);
  load_tables(K, s);
  __syncthreads();
  const int tid = threadIdx.x, NP = K.NP;
  double acc = 0.0;
  for (int c = blockIdx.x; c < L.ncell; c += gridDim.x) {
    const int i = c % L.nx, j = c / L.nx;
    double loc = 0.0;
    if (mode == kResOut || mode == kResDefectNorm) {
      cell_residual<false, false, kES>(K, L, s, i, j, [&](int o, double Rr) {
        if (mode == kResDefectNorm)
          L.D[(size_t)c * NP + o] = -Rr;
        else if (out)
          out[(size_t)c * out_stride + o] = Rr;
        double w = s.fact[o] * s.sc[S_TPOW + s.tdeg[o]];
        loc += w * Rr * Rr;
      });
      if (out && mode == kResOut)  // planar: the rows with odd alpha_3 are exactly zero
        for (int o = tid; o < K.N; o += kThreads)
          if (s.tal[2 * K.N + o] & 1) out[(size_t)c * out_stride + o] = 0.0;
      double t = block_sum(loc, s.sc + S_RED);
      if (tid == 0) acc += L.uniform ? t * L.dx * L.dy : t * (L.hx[i] * L.hy[j]);
    } else if (mode == kResDefect) {
      cell_residual<false, false, kES>(K, L, s, i, j, [&](int o, double Rr) { L.D[(size_t)c * NP + o] = -Rr; });
    } else {
      cell_residual<false, false, kES>(K, L, s, i, j,
                           [&](int o, double Rr) { L.rF[(size_t)c * NP + o] = Rr + L.rF[(size_t)c * NP + o]; });
    }
    __syncthreads();
  }
  if (tid == 0 && partials) partials[blockIdx.x] = acc;
}

// ------------------------------------------------------------------ restriction (Sec. 3.2.2)
__global__ void __launch_bounds__(kThreads) restrict_kernel(Consts K, LevelDev Lf, LevelDev Lc) {
  extern __shared__ __align__(16) char smem_raw[];
  Sm s = bind_smem(smem_raw, K.M, K.N, K.NP);
  load_tables(K, s);
  __syncthreads();
  const int tid = threadIdx.x, NE = K.NE, NP = K.NP;
  for (int C = blockIdx.x; C < Lc.ncell; C += gridDim.x) {
    const int I = C % Lc.nx, J = C / Lc.nx;
    int fi[4] = {(2 * J) * Lf.nx + 2 * I, (2 * J) * Lf.nx + 2 * I + 1, (2 * J + 1) * Lf.nx + 2 * I,
                 (2 * J + 1) * Lf.nx + 2 * I + 1};
    // fine states into VA slots 0..3, fine defects into slots 4..7 (even alpha_3 only)
    for (int q = tid; q < 8 * NE; q += kThreads) {
      int v = q / NE, o = s.eidx[q - v * NE];
      int cc = fi[v & 3];
      s.VA[v * NP + o] = v < 4 ? Lf.F[(size_t)cc * NP + o] : Lf.D[(size_t)cc * NP + o];
    }
    if (tid < 32) {
      int v = tid >> 2, e = tid & 3;
      s.vsrc[v * 4 + e] = Lf.P[(size_t)fi[v & 3] * 4 + e];
    }
    __syncthreads();
    if (tid == 0) {
      // (u_H, theta_H) from conservation of mass, momentum and energy (eq. uH-thetaH-computation)
      // children's area weights (equal areas: 1 each, then the plain mean)
      const double mean = Lf.uniform ? 0.25 : 1.0;
      for (int q = 0; q < 4; ++q)
        s.sc[S_W + q] = Lf.uniform ? 1.0
                                   : Lf.hx[fi[q] % Lf.nx] * Lf.hy[fi[q] / Lf.nx] / (Lc.hx[I] * Lc.hy[J]);
      double rho = 0.0, mom[3] = {0.0, 0.0, 0.0}, en = 0.0;
      for (int q = 0; q < 4; ++q) {
        const double *p = s.vsrc + q * 4;
        double r = s.sc[S_W + q] * s.VA[q * NP];
        rho += r;
        for (int d = 0; d < 3; ++d) mom[d] += r * p[d];
        en += r * (p[0] * p[0] + p[1] * p[1] + p[2] * p[2]) + 3.0 * r * p[3];
      }
      rho *= mean;
      for (int d = 0; d < 3; ++d) mom[d] *= mean;
      en *= mean;
      double *pH = s.sc + S_PH;
      for (int d = 0; d < 3; ++d) pH[d] = mom[d] / rho;
      pH[3] = (en - rho * (pH[0] * pH[0] + pH[1] * pH[1] + pH[2] * pH[2])) / (3.0 * rho);
      s.sc[S_TPN] = pow(pH[3], 1.0 - K.omega);
      for (int v = 0; v < 8; ++v) {
        for (int e = 0; e < 4; ++e) s.vdst[v * 4 + e] = pH[e];
        s.iarr[I_ACT + v] = v;
      }
      s.iarr[I_NACT] = 8;
    }
    __syncthreads();
    setup_coeffs(K, s);
    __syncthreads();
    transform_batch(K, s, s.VA, s.VB);
    // area means (eq. fH)
    double *fH = s.VA, *RH = s.VA + NP;
    for (int q = tid; q < NE; q += kThreads) {
      const int o = s.eidx[q];
      double a = 0.0, b = 0.0;
      if (Lf.uniform) {
        for (int q = 0; q < 4; ++q) {
          a += s.VB[q * NP + o];
          b += s.VB[(4 + q) * NP + o];
        }
        a *= 0.25;
        b *= 0.25;
      } else {
        for (int q = 0; q < 4; ++q) {
          a += s.sc[S_W + q] * s.VB[q * NP + o];
          b += s.sc[S_W + q] * s.VB[(4 + q) * NP + o];
        }
      }
      fH[o] = a;
      RH[o] = b;
    }
    __syncthreads();
    if (tid == 0) {
      for (int d = 0; d < 2; ++d) fH[K.idx_e[d]] = 0.0;
      double s3 = (fH[K.idx_2e[0]] + fH[K.idx_2e[1]] + fH[K.idx_2e[2]]) * (1.0 / 3.0);
      for (int d = 0; d < 3; ++d) fH[K.idx_2e[d]] -= s3;
    }
    __syncthreads();
    for (int q = tid; q < NE; q += kThreads) {
      const int o = s.eidx[q];
      Lc.F[(size_t)C * NP + o] = fH[o];
      Lc.bF[(size_t)C * NP + o] = fH[o];
      Lc.rF[(size_t)C * NP + o] = RH[o];
    }
    if (tid < 4) {
      double v = s.sc[S_PH + tid];
      Lc.P[(size_t)C * 4 + tid] = v;
      Lc.bP[(size_t)C * 4 + tid] = v;
      Lc.rP[(size_t)C * 4 + tid] = v;
    }
    if (tid == 4) Lc.tp[C] = s.sc[S_TPN];
    __syncthreads();
  }
}

// ------------------------------------------------------------------ coarse-grid update (eq. rewritten-update)
__global__ void __launch_bounds__(kThreads) prolong_kernel(Consts K, LevelDev Lf, LevelDev Lc) {
  extern __shared__ __align__(16) char smem_raw[];
  Sm s = bind_smem(smem_raw, K.M, K.N, K.NP);
  load_tables(K, s);
  __syncthreads();
  const int tid = threadIdx.x, NE = K.NE, NP = K.NP;
  for (int c = blockIdx.x; c < Lf.ncell; c += gridDim.x) {
    const int i = c % Lf.nx, j = c / Lf.nx;
    const int C = (j / 2) * Lc.nx + i / 2;
    // slot 1: restricted coarse state, slot 2: current coarse state, both into the fine basis
    for (int q = tid; q < 2 * NE; q += kThreads) {
      int v = q / NE, o = s.eidx[q - v * NE];
      s.VA[(1 + v) * NP + o] = v == 0 ? Lc.bF[(size_t)C * NP + o] : Lc.F[(size_t)C * NP + o];
    }
    if (tid < 8) {
      int v = tid >> 2, e = tid & 3;
      s.vsrc[(1 + v) * 4 + e] = v == 0 ? Lc.bP[(size_t)C * 4 + e] : Lc.P[(size_t)C * 4 + e];
      s.vdst[(1 + v) * 4 + e] = Lf.P[(size_t)c * 4 + e];
    }
    if (tid < 4) s.sc[S_PH + tid] = Lf.P[(size_t)c * 4 + tid];
    if (tid == 0) {
      s.iarr[I_ACT] = 1;
      s.iarr[I_ACT + 1] = 2;
      s.iarr[I_NACT] = 2;
    }
    __syncthreads();
    setup_coeffs(K, s);
    __syncthreads();
    transform_batch(K, s, s.VA, s.VB);
    for (int q = tid; q < NE; q += kThreads) {
      const int o = s.eidx[q];
      s.VA[o] = (Lf.F[(size_t)c * NP + o] - s.VB[1 * NP + o]) + s.VB[2 * NP + o];
    }
    __syncthreads();
    double pcell[4];
    for (int e = 0; e < 4; ++e) pcell[e] = s.sc[S_PH + e];
    bool ok = regrad(K, s, pcell, 0, true);
    for (int q = tid; q < NE; q += kThreads) {
      const int o = s.eidx[q];
      Lf.F[(size_t)c * NP + o] = s.VB[o];
    }
    if (tid < 4) Lf.P[(size_t)c * 4 + tid] = s.sc[S_NEWP + tid];
    if (tid == 4) Lf.tp[c] = s.sc[S_TPN];
    if (!ok && tid == 0) raise_status(K, kStNonPhysical, false);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ forward Euler (Sec. 2.4)
// The level's step of eq. (global-CFL): the smallest local step of eq. (local-CFL) over the
// level (each capped at dtnu / nu when dtnu > 0), reduced by one block.
__global__ void euler_dt_kernel(Consts K, LevelDev L, double *dt_out) {
  __shared__ double red[kThreads];
  double m = INFINITY;
  for (int c = threadIdx.x; c < L.ncell; c += kThreads) {
    const double *p = L.P + (size_t)c * 4;
    const double sq = sqrt(p[3]);
    const int ci = c % L.nx, cj = c / L.nx;
    double dt = K.cfl / ((fabs(p[0]) + K.C * sq) * inv_hx(L, ci) + (fabs(p[1]) + K.C * sq) * inv_hy(L, cj));
    if (K.dtnu > 0.0) dt = fmin(dt, K.dtnu / (K.nu0 * L.F[(size_t)c * K.NP] * L.tp[c]));
    m = fmin(m, dt);
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) dt_out[0] = red[0];
}

// eq. (euler-scheme): f <- Grad(f + dt (R(f) - r)) for every cell, with R - r of the old state
// in L.D (written by the residual kernel before any cell changes) and dt from euler_dt_kernel.
__global__ void __launch_bounds__(kThreads) euler_update_kernel(Consts K, LevelDev L, const double *dt_in) {
  extern __shared__ __align__(16) char smem_raw[];
  Sm s = bind_smem(smem_raw, K.M, K.N, K.NP);
  load_tables(K, s);
  __syncthreads();
  const int tid = threadIdx.x, NE = K.NE, NP = K.NP;
  const double dt = *dt_in;
  for (int c = blockIdx.x; c < L.ncell; c += gridDim.x) {
    for (int q = tid; q < NE; q += kThreads) {
      const int o = s.eidx[q];
      s.VA[o] = fma(dt, L.D[(size_t)c * NP + o], L.F[(size_t)c * NP + o]);
    }
    if (tid < 4) s.sc[S_PH + tid] = L.P[(size_t)c * 4 + tid];
    __syncthreads();
    double pcell[4];
    for (int e = 0; e < 4; ++e) pcell[e] = s.sc[S_PH + e];
    bool ok = regrad(K, s, pcell, 0, true);
    for (int q = tid; q < NE; q += kThreads) {
      const int o = s.eidx[q];
      L.F[(size_t)c * NP + o] = s.VB[o];
    }
    if (tid < 4) L.P[(size_t)c * 4 + tid] = s.sc[S_NEWP + tid];
    if (tid == 4) L.tp[c] = s.sc[S_TPN];
    if (!ok && tid == 0) raise_status(K, kStNonPhysical, false);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ reductions and small kernels
__global__ void reduce_norm_kernel(const double *partials, int n, double scale, double *out) {
  __shared__ double red[kThreads / 32];
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += kThreads) v += partials[k];
  double t = block_sum(v, red);
  if (threadIdx.x == 0) out[0] = sqrt(t * scale);
}

__global__ void mass_partial_kernel(LevelDev L, int NP, double *partials) {
  __shared__ double red[kThreads / 32];
  double v = 0.0;
  for (int c = blockIdx.x * kThreads + threadIdx.x; c < L.ncell; c += gridDim.x * kThreads)
    v += L.uniform ? L.F[(size_t)c * NP] : L.F[(size_t)c * NP] * cell_area(L, c % L.nx, c / L.nx);
  double t = block_sum(v, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// total mass sum_c rho_c * area into out[0]; the scale m0 / mass into out[1] when m0 > 0
__global__ void mass_total_kernel(const double *partials, int n, double area, double m0, double *out) {
  __shared__ double red[kThreads / 32];
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += kThreads) v += partials[k];
  double t = block_sum(v, red);
  if (threadIdx.x == 0) {
    out[0] = t * area;
    if (m0 > 0.0) out[1] = m0 / (t * area);
  }
}

__global__ void mass_apply_kernel(LevelDev L, int NP, const double *scale) {
  const double sc = scale[0];
  size_t tot = (size_t)L.ncell * NP;
  for (size_t q = (size_t)blockIdx.x * kThreads + threadIdx.x; q < tot; q += (size_t)gridDim.x * kThreads)
    L.F[q] *= sc;
}

// Grad-basis fields (eq. moments-relation): rho, u, theta, sigma_ij = (1+delta_ij) f_{e_i+e_j},
// q_i = 2 f_{3e_i} + sum_d f_{2e_d+e_i}.  The needed indices sit after the Shakhov table.
__global__ void fields_kernel(Consts K, LevelDev L, double *out) {
  for (int c = blockIdx.x * kThreads + threadIdx.x; c < L.ncell; c += gridDim.x * kThreads) {
    const double *f = L.F + (size_t)c * K.NP, *p = L.P + (size_t)c * 4;
    const int *iq = K.tab_i32 + K.iq_off;       // [3][4] heat-flux indices
    const int *is = K.tab_i32 + K.iq_off + 12;  // [6] idx(e_i + e_j), i <= j
    double *o = out + (size_t)c * 14;
    o[0] = f[0];
    for (int d = 0; d < 3; ++d) o[1 + d] = p[d];
    o[4] = p[3];
    int k = 0;
    for (int a = 0; a < 3; ++a)
      for (int b = a; b < 3; ++b, ++k) o[5 + k] = (1.0 + (a == b)) * f[is[k]];
    for (int a = 0; a < 3; ++a) {
      double q = 2.0 * f[iq[4 * a]];
      for (int d = 0; d < 3; ++d) q += f[iq[4 * a + 1 + d]];
      o[11 + a] = q;
    }
  }
}

__global__ void tpow_kernel(Consts K, LevelDev L) {
  for (int c = blockIdx.x * kThreads + threadIdx.x; c < L.ncell; c += gridDim.x * kThreads)
    L.tp[c] = pow(L.P[(size_t)c * 4 + 3], 1.0 - K.omega);
}

__global__ void pack_kernel(const double *src, int ss, double *dst, int ds, int rows, int cols) {
  size_t tot = (size_t)rows * ds;
  for (size_t q = (size_t)blockIdx.x * kThreads + threadIdx.x; q < tot; q += (size_t)gridDim.x * kThreads) {
    size_t r = q / ds;
    int col = (int)(q - r * ds);
    dst[q] = col < cols ? src[r * ss + col] : 0.0;
  }
}

// Admissibility of a state (rhs = 0: rho > 0, theta > 0) or of a right-hand side (rhs = 1:
// theta > 0) handed in through the C ABI: finite, and planar (u_3 = 0, odd alpha_3 zero).
__global__ void check_state_kernel(Consts K, const double *P, const double *F, int stride, int ncell, int rhs) {
  const uint16_t *a3 = K.tab_u16 + 9 * K.N + 2 * K.N;
  for (int c = blockIdx.x * kThreads + threadIdx.x; c < ncell; c += gridDim.x * kThreads) {
    const double *p = P + (size_t)c * 4, *f = F + (size_t)c * stride;
    bool ok = isfinite(p[0]) && isfinite(p[1]) && isfinite(p[3]) && p[3] > 0.0 && (rhs || f[0] > 0.0);
    bool planar = p[2] == 0.0;
    for (int o = 0; o < K.N; ++o) {
      ok = ok && isfinite(f[o]);
      if (a3[o] & 1) planar = planar && f[o] == 0.0;
    }
    if (!planar) atomicCAS(K.status, 0, 1);
    if (!ok) atomicCAS(K.status, 0, kStNonPhysical);
  }
}

// ------------------------------------------------------------------ launchers
static void init_attrs() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(fs_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  cudaFuncSetAttribute(fs_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  cudaFuncSetAttribute(fs_cluster_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  cudaFuncSetAttribute(fs_cluster_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  cudaFuncSetAttribute(residual_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  cudaFuncSetAttribute(residual_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  cudaFuncSetAttribute(restrict_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  cudaFuncSetAttribute(prolong_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  cudaFuncSetAttribute(euler_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  done = true;
}
template <typename Kern>
static void ensure_smem_attr(Kern) {
  init_attrs();
}

static size_t smem_for(const Consts &K) { return make_layout(K.M, K.N, K.NP).total; }

cudaError_t launch_fs(const Consts &K, const LevelDev &L, int steps, const int *queue, int grid, cudaStream_t st) {
  init_attrs();
  if (K.model == 2)
    fs_kernel<true><<<grid, kThreads, smem_for(K), st>>>(K, L, steps, queue);
  else
    fs_kernel<false><<<grid, kThreads, smem_for(K), st>>>(K, L, steps, queue);
  return cudaGetLastError();
}

static cudaLaunchConfig_t cluster_config(const Consts &K, int nclusters, int per_sm, cudaStream_t st,
                                         cudaLaunchAttribute *attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * nclusters, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = std::max(cluster_smem_bytes(K.M, K.N, K.NP), kClusterMinSmem[per_sm > 1 ? 1 : 0]);
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

cudaError_t launch_fs_cluster(const Consts &K, const LevelDev &L, int steps, const int *queue, int nclusters,
                              int per_sm, cudaStream_t st) {
  init_attrs();
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_config(K, nclusters, per_sm, st, attr);
  if (K.model == 2) return cudaLaunchKernelEx(&cfg, fs_cluster_kernel<true>, K, L, steps, queue);
  return cudaLaunchKernelEx(&cfg, fs_cluster_kernel<false>, K, L, steps, queue);
}

int cluster_capacity(const Consts &K, int per_sm) {
  init_attrs();
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_config(K, 1, per_sm, nullptr, attr);
  int n = 0;
  cudaError_t e = K.model == 2 ? cudaOccupancyMaxActiveClusters(&n, fs_cluster_kernel<true>, &cfg)
                               : cudaOccupancyMaxActiveClusters(&n, fs_cluster_kernel<false>, &cfg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_fs_batch(const BatchDesc *desc, const int2 *items, long long total, int *counter,
                            const Consts &K0, int grid, cudaStream_t st) {
  static bool done = false;
  if (!done) {
    // the descriptor copy is static shared memory: the dynamic part gets the rest
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fs_batch_kernel<false>);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fs_batch_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024 - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncGetAttributes(&fa, fs_batch_kernel<true>);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fs_batch_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024 - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
    done = true;
  }
  if (K0.model == 2)
    fs_batch_kernel<true><<<grid, kThreads, smem_for(K0), st>>>(desc, items, total, counter, K0);
  else
    fs_batch_kernel<false><<<grid, kThreads, smem_for(K0), st>>>(desc, items, total, counter, K0);
  return cudaGetLastError();
}

cudaError_t launch_residual(const Consts &K, const LevelDev &L, int mode, double *out, int out_stride,
                            double *partials, int grid, cudaStream_t st) {
  init_attrs();
  if (K.model == 2)
    residual_kernel<true><<<grid, kThreads, smem_for(K), st>>>(K, L, mode, out, out_stride, partials);
  else
    residual_kernel<false><<<grid, kThreads, smem_for(K), st>>>(K, L, mode, out, out_stride, partials);
  return cudaGetLastError();
}

cudaError_t launch_restrict(const Consts &K, const LevelDev &Lf, const LevelDev &Lc, int grid, cudaStream_t st) {
  ensure_smem_attr(restrict_kernel);
  restrict_kernel<<<grid, kThreads, smem_for(K), st>>>(K, Lf, Lc);
  return cudaGetLastError();
}

cudaError_t launch_prolong(const Consts &K, const LevelDev &Lf, const LevelDev &Lc, int grid, cudaStream_t st) {
  ensure_smem_attr(prolong_kernel);
  prolong_kernel<<<grid, kThreads, smem_for(K), st>>>(K, Lf, Lc);
  return cudaGetLastError();
}

cudaError_t launch_euler(const Consts &K, const LevelDev &L, double *dt_dev, int grid, cudaStream_t st) {
  init_attrs();
  euler_dt_kernel<<<1, kThreads, 0, st>>>(K, L, dt_dev);
  euler_update_kernel<<<grid, kThreads, smem_for(K), st>>>(K, L, dt_dev);
  return cudaGetLastError();
}

cudaError_t launch_reduce_norm(const double *partials, int n, double scale, double *out, cudaStream_t st) {
  reduce_norm_kernel<<<1, kThreads, 0, st>>>(partials, n, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_mass(const Consts &K, const LevelDev &L, double *partials, int grid, double *scal, double m0,
                        bool apply, cudaStream_t st) {
  mass_partial_kernel<<<grid, kThreads, 0, st>>>(L, K.NP, partials);
  // a uniform grid sums rho and scales by the common cell area; otherwise the partials hold
  // rho times each cell's area
  mass_total_kernel<<<1, kThreads, 0, st>>>(partials, grid, L.uniform ? L.dx * L.dy : 1.0, m0, scal);
  if (apply) {
    int g2 = (int)(((size_t)L.ncell * K.NP + kThreads - 1) / kThreads);
    if (g2 > 4096) g2 = 4096;
    mass_apply_kernel<<<g2, kThreads, 0, st>>>(L, K.NP, scal + 1);
  }
  return cudaGetLastError();
}

cudaError_t launch_fields(const Consts &K, const LevelDev &L, double *out, cudaStream_t st) {
  int g = (L.ncell + kThreads - 1) / kThreads;
  if (g > 4096) g = 4096;
  fields_kernel<<<g, kThreads, 0, st>>>(K, L, out);
  return cudaGetLastError();
}

cudaError_t launch_tpow(const Consts &K, const LevelDev &L, cudaStream_t st) {
  int g = (L.ncell + kThreads - 1) / kThreads;
  if (g > 4096) g = 4096;
  tpow_kernel<<<g, kThreads, 0, st>>>(K, L);
  return cudaGetLastError();
}

cudaError_t launch_pack(const double *src, int src_stride, double *dst, int dst_stride, int rows, int cols,
                        cudaStream_t st) {
  size_t tot = (size_t)rows * dst_stride;
  int g = (int)((tot + kThreads - 1) / kThreads);
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  pack_kernel<<<g, kThreads, 0, st>>>(src, src_stride, dst, dst_stride, rows, cols);
  return cudaGetLastError();
}

cudaError_t launch_check_state(const Consts &K, const double *P, const double *F, int stride, int ncell, int rhs,
                               cudaStream_t st) {
  int g = (ncell + kThreads - 1) / kThreads;
  if (g > 4096) g = 4096;
  check_state_kernel<<<g, kThreads, 0, st>>>(K, P, F, stride, ncell, rhs);
  return cudaGetLastError();
}

int occupancy_cell(int M, int NP, int which) {
  int N = (M + 1) * (M + 2) * (M + 3) / 6;
  size_t sm = make_layout(M, N, NP).total;
  int nb = 0;
  switch (which) {
    case 0: {  // the smaller of the two instantiations' occupancies
      init_attrs();
      int nb2 = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fs_kernel<false>, kThreads, sm);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb2, fs_kernel<true>, kThreads, sm);
      nb = std::min(nb, nb2);
      break;
    }
    case 1: {
      init_attrs();
      int nb2 = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, residual_kernel<false>, kThreads, sm);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb2, residual_kernel<true>, kThreads, sm);
      nb = std::min(nb, nb2);
      break;
    }
    case 2:
      ensure_smem_attr(restrict_kernel);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, restrict_kernel, kThreads, sm);
      break;
    default:
      ensure_smem_attr(prolong_kernel);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, prolong_kernel, kThreads, sm);
      break;
  }
  return nb;
}

}  // namespace nrmg
