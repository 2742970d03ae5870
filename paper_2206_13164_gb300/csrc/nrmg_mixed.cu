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
//
// The correction sweep is bound by the latency of the chain of dependent cell updates, not by
// FP32 arithmetic.  Two things keep global-memory round trips off that chain: each correction
// coefficient travels in one 64-bit word together with the version of the update that wrote it
// (so the data is its own ready flag: no release fence, no flag load before the data load), and
// everything that stays fixed during the launch (frozen coefficients, FP32 state, the defect) is
// copied into shared memory asynchronously while the dependencies are still pending.
#include "nrmg_device.cuh"

namespace nrmg {

// ------------------------------------------------------------------ shared-memory layout (FP32)
struct CLayout {
  size_t cst, VA, VB, ss, dd, vsrc, vdst, cf, sc, ti32, vflag, iarr, tu16, wl, total;
};
// Longest index line of the line-wise transform (M <= kLineMax - 1; higher orders use the
// output-wise transform_batch of the FP64 path).
constexpr int kLineMax = 11;
// Row stride of the transform vectors in shared memory: NP + 1 for the line-wise transform, so
// that the lanes that take one index line of several vectors hit distinct banks (NP is a
// multiple of 4, and of 32 for some orders); NP for transform_batch.
__host__ __device__ inline int corr_vstride(int M, int NP) { return M < kLineMax ? NP + 1 : NP; }
// FP32 wall tables in shared memory: W [4][(M+1)^2], rho weights [4][M+1], incoming [4][M+1]
__host__ __device__ inline int wall_floats(int M) { return 4 * (M + 1) * (M + 1) + 8 * (M + 1); }

__host__ __device__ inline CLayout make_corr_layout(int M, int N, int NP) {
  const int NE = nmom_even(M);
  CLayout s;
  size_t o = 0;
  size_t vb = (size_t)8 * (8 + NP), va = (size_t)kNV * corr_vstride(M, NP);
  if (va > vb) vb = va;
  s.cst = o;   o = al16(o + sizeof(float) * (8 + NP));
  s.VA = o;    o = al16(o + sizeof(float) * va);
  s.VB = o;    o = al16(o + sizeof(float) * vb);
  s.ss = o;    o = al16(o + sizeof(float) * 9 * NP);
  s.dd = o;    o = al16(o + sizeof(float) * NP);
  s.vsrc = o;  o = al16(o + sizeof(float) * kNV * 4);
  s.vdst = o;  o = al16(o + sizeof(float) * kNV * 4);
  s.cf = o;    o = al16(o + sizeof(float) * kNV * 3 * (M + 1));
  s.sc = o;    o = al16(o + sizeof(float) * 64);
  s.ti32 = o;  o = al16(o + sizeof(int) * (3 * NE + N + 18 + nlines_total(M)));
  s.vflag = o; o = al16(o + sizeof(int) * kNV * 3);
  s.iarr = o;  o = al16(o + sizeof(int) * 64);
  s.tu16 = o;  o = al16(o + sizeof(uint16_t) * (13 * N + NE));
  s.wl = o;    o = al16(o + sizeof(float) * wall_floats(M));
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
// the updated cell's FP32 defect row
__device__ inline float *corr_defect(char *base, int M, int N, int NP) {
  return (float *)(base + make_corr_layout(M, N, NP).dd);
}

// ------------------------------------------------------------------ tagged correction words
// Each coefficient of the correction is one 64-bit word: the FP32 value in the low half, the
// version of the update that wrote it in the high half.  A naturally aligned 64-bit access is
// single-copy atomic, so a reader that sees the version it needs also sees that update's value:
// the word itself is the flag, and neither a fence on the writer's side nor a separate flag
// load on the reader's side sits between two dependent updates.
__device__ inline unsigned long long ld_relaxed_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ inline void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ inline unsigned long long tag_word(float x, int version) {
  return ((unsigned long long)(unsigned)version << 32) | (unsigned long long)__float_as_uint(x);
}
__device__ inline int word_version(unsigned long long w) { return (int)(unsigned)(w >> 32); }
__device__ inline float word_value(unsigned long long w) { return __uint_as_float((unsigned)w); }

// 16-byte asynchronous copy global -> shared (both addresses 16-byte aligned)
__device__ inline void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// One warp copies the even-alpha_3 entries of a cell's correction row (src, NP words) into
// dst once each word carries version `need` or newer.  Every lane keeps its unsatisfied words
// and re-reads them (the loop is warp-uniform); lane 0 watches the abort flag and the time
// limit.  Returns false when the wait gave up.
__device__ inline bool ll_row(const Consts &K, const uint16_t *eidx, const unsigned long long *src, float *dst,
                              int need, int lane) {
  constexpr int kU = 8;
  const int NE = K.NE;
  unsigned long long t0 = 0;
  for (int b = 0; b < NE; b += kU * 32) {
    unsigned long long w[kU];
    int o[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = b + lane + u * 32;
      o[u] = e < NE ? (int)eidx[e] : -1;
      if (o[u] >= 0) w[u] = ld_relaxed_u64(src + o[u]);
    }
    unsigned pend = 0;
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (o[u] >= 0) {
        if (word_version(w[u]) >= need)
          dst[o[u]] = word_value(w[u]);
        else
          pend |= 1u << u;
      }
    for (int it = 0; __any_sync(0xffffffffu, pend != 0); ++it) {
      // the time limit is checked on every round, the abort word (a global load) on every
      // 16th, so that a round costs one load latency
      int stop = 0;
      if (lane == 0) {
        if (t0 == 0) t0 = gtimer();
        if ((it & 15) == 15 && ld_volatile(K.abort_flag)) {
          stop = 1;
        } else if (gtimer() - t0 > kWaitLimitNs) {
          raise_status(K, kStTimeout, true);
          stop = 1;
        }
      }
      if (__shfl_sync(0xffffffffu, stop, 0)) return false;
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if ((pend >> u) & 1u) {
          const unsigned long long x = ld_relaxed_u64(src + o[u]);
          if (word_version(x) >= need) {
            dst[o[u]] = word_value(x);
            pend &= ~(1u << u);
          }
        }
    }
  }
  return true;
}

// half of the limited slope of the frozen face bases (FP32 twin of the FP64 reconstruction)
__device__ inline float half_slope_f(int slope, float qm, float q0, float qp) {
  if (slope == 1) return 0.25f * (qp - qm);
  float a = q0 - qm, b = qp - q0;
  // the linearized operator only needs the weights approximately: fast division
  return __fdividef(0.5f * ((a + b) * fmaf(a, b, 1e-12f)), fmaf(a, a, fmaf(b, b, 2e-12f)));
}

enum { C_DT = 0, C_NU = 1, C_Q = 2 /* ..5 */, C_W = 8 /* ..8+12 */, C_RHOW = 20 /* ..24 */ };

// ------------------------------------------------------------------ line-wise FP32 basis transform
// g = prod_d exp(-a_d S_d - b S_d^2) f for the active vectors, as the FP64 transform, but with
// one thread per (vector, index line): the thread holds the line's inputs and the direction's
// series coefficients in registers and forms every output of the line, y_n = sum_{k<=n} c_k
// x_{n-k} (n = position along the line), so no output waits on a chain of shared-memory index
// loads.  Along alpha_3 only the even entries take part: a_3 = 0 for planar states, so the odd
// coefficients c_k vanish and even outputs only see even inputs.  Lines are ordered longest
// first; passes X->Y, Y->X, X->Y.
// One index line along x or y per lane, the warp's lines at most kL long (L <= kL per lane,
// 0 for an idle lane): inputs, indices and series coefficients in registers; every lane runs
// the same kL-long code (entries from L on are zero and their outputs are not stored), so the
// warp never diverges on the line length.  Each output sums its terms in two partial sums in
// ascending k, as transform_one does (a nonzero a: odd k in the first, even k >= 2 in the
// second; a = 0: the odd c_k vanish, k = 2 mod 4 goes to the first, k = 0 mod 4 to the
// second), so both transforms round alike; a warp takes the second ordering only when one of
// its lanes has a = 0.  An identity transform (a = b = 0) adds exact zeros.
template <int kL>
__device__ __forceinline__ void line_xy(const float *x, float *y, const float *c, const uint16_t *m, int L, int fl,
                                        bool any_zero_a) {
  float a0[kL], a1[kL], xv[kL];
  int id[kL];
  const bool ident = fl & 1, zero_a = (fl & 2) && !ident;
#pragma unroll
  for (int q = 0; q < kL; ++q) id[q] = q < L ? (int)m[q] : -1;
#pragma unroll
  for (int q = 0; q < kL; ++q) {
    xv[q] = id[q] >= 0 ? x[id[q]] : 0.0f;
    a0[q] = xv[q];
    a1[q] = 0.0f;
  }
  if (!any_zero_a) {
#pragma unroll
    for (int k = 1; k < kL; ++k) {
      const float ck = (ident || k >= L) ? 0.0f : c[k];
#pragma unroll
      for (int n = k; n < kL; ++n) {
        if (k & 1)
          a0[n] = fmaf(ck, xv[n - k], a0[n]);
        else
          a1[n] = fmaf(ck, xv[n - k], a1[n]);
      }
    }
  } else {
#pragma unroll
    for (int k = 1; k < kL; ++k) {
      const float ck = (ident || k >= L) ? 0.0f : c[k];
      const bool first = zero_a ? (k & 3) == 2 : (k & 1);
#pragma unroll
      for (int n = k; n < kL; ++n) {
        const float t = fmaf(ck, xv[n - k], first ? a0[n] : a1[n]);
        if (first)
          a0[n] = t;
        else
          a1[n] = t;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kL; ++q)
    if (id[q] >= 0) y[id[q]] = a0[q] + a1[q];
}

// Along alpha_3 (at most kE even entries per lane, alpha_3 = 2n at position 2n of the line):
// c_{2j} with j odd in the first partial sum, j even in the second.
template <int kE>
__device__ __forceinline__ void line_z(const float *x, float *y, const float *c, const uint16_t *m, int Le, int fl) {
  float a0[kE], a1[kE], xv[kE];
  int id[kE];
  const bool ident = fl & 1;
#pragma unroll
  for (int q = 0; q < kE; ++q) id[q] = q < Le ? (int)m[2 * q] : -1;
#pragma unroll
  for (int q = 0; q < kE; ++q) {
    xv[q] = id[q] >= 0 ? x[id[q]] : 0.0f;
    a0[q] = xv[q];
    a1[q] = 0.0f;
  }
#pragma unroll
  for (int k = 1; k < kE; ++k) {
    const float ck = (ident || k >= Le) ? 0.0f : c[2 * k];
#pragma unroll
    for (int n = k; n < kE; ++n) {
      if (k & 1)
        a0[n] = fmaf(ck, xv[n - k], a0[n]);
      else
        a1[n] = fmaf(ck, xv[n - k], a1[n]);
    }
  }
#pragma unroll
  for (int q = 0; q < kE; ++q)
    if (id[q] >= 0) y[id[q]] = a0[q] + a1[q];
}

// g = prod_d exp(-a_d S_d - b S_d^2) f for the active vectors, as the FP64 transform, but with
// one lane per (index line, vector): the lane holds the line's inputs and the direction's
// series coefficients in registers and forms every output of the line, y_n = sum_{k<=n} c_k
// x_{n-k} (n = position along the line), so no output waits on a chain of shared-memory index
// loads.  Along alpha_3 only the even entries take part: a_3 = 0 for planar states, so the odd
// coefficients c_k vanish and even outputs only see even inputs.  Lines are ordered longest
// first and consecutive lanes take one line of consecutive vectors, so a warp's lines have
// similar lengths; the warp runs the code of its longest line.  Passes X->Y, Y->X, X->Y;
// vectors VS floats apart.
__device__ __forceinline__ void transform_lines(const Consts &K, SmT<float> &s, const int *lines, float *X, float *Y,
                                             int VS) {
  const int N = K.N, M = K.M, na = s.iarr[I_NACT];
  const int lane = threadIdx.x & 31;
  const int *ln = lines;
  for (int d = 0; d < 3; ++d) {
    const float *in = (d == 1) ? Y : X;
    float *out = (d == 1) ? X : Y;
    const int nl = K.nl[d], tot = na * nl;
    const uint16_t *mem = s.tmem + d * N;
    for (int tb = threadIdx.x - lane; tb < tot; tb += kThreads) {  // warp-uniform loop
      const int t = tb + lane;
      int L = 0, fl = 1, v = 0;
      const uint16_t *m = mem;
      if (t < tot) {
        const int l = t / na, vi = t - l * na;
        v = s.iarr[I_ACT + vi];
        const int code = ln[l];
        L = code >> 11;
        m = mem + (code & 2047);
        fl = s.vflag[v * 3 + d];
      }
      const float *c = s.cf + (v * 3 + d) * (M + 1);
      const float *x = in + v * VS;
      float *y = out + v * VS;
      if (d < 2) {
        const int Lw = __reduce_max_sync(0xffffffffu, (unsigned)L);
        const bool anyz = __any_sync(0xffffffffu, (fl & 2) && !(fl & 1) && L > 0);
        switch (Lw) {
          case 0: break;
          case 1: line_xy<1>(x, y, c, m, L, fl, anyz); break;
          case 2: line_xy<2>(x, y, c, m, L, fl, anyz); break;
          case 3: line_xy<3>(x, y, c, m, L, fl, anyz); break;
          case 4: line_xy<4>(x, y, c, m, L, fl, anyz); break;
          case 5: line_xy<5>(x, y, c, m, L, fl, anyz); break;
          case 6: line_xy<6>(x, y, c, m, L, fl, anyz); break;
          case 7: line_xy<7>(x, y, c, m, L, fl, anyz); break;
          case 8: line_xy<8>(x, y, c, m, L, fl, anyz); break;
          case 9: line_xy<9>(x, y, c, m, L, fl, anyz); break;
          case 10: line_xy<10>(x, y, c, m, L, fl, anyz); break;
          default: line_xy<11>(x, y, c, m, L, fl, anyz); break;
        }
      } else {
        const int Le = (L + 1) >> 1;
        switch (__reduce_max_sync(0xffffffffu, (unsigned)Le)) {
          case 0: break;
          case 1: line_z<1>(x, y, c, m, Le, fl); break;
          case 2: line_z<2>(x, y, c, m, Le, fl); break;
          case 3: line_z<3>(x, y, c, m, Le, fl); break;
          case 4: line_z<4>(x, y, c, m, Le, fl); break;
          case 5: line_z<5>(x, y, c, m, Le, fl); break;
          default: line_z<6>(x, y, c, m, Le, fl); break;
        }
      }
    }
    ln += nl;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ frozen coefficients and FP32 defect
__global__ void mixed_prep_kernel(Consts K, LevelDev L) {
  const size_t tot = (size_t)L.ncell * K.NP;
  for (size_t q = (size_t)blockIdx.x * kThreads + threadIdx.x; q < tot; q += (size_t)gridDim.x * kThreads) {
    L.d32[q] = (float)L.D[q];
    L.et[q] = 0ull;  // e = 0, version 0
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
  // constant tables: index tables and lines, the FP32 wall tables
  const int ni32 = K.ln_off + nlines_total(M);
  for (int e = tid; e < ni32; e += kThreads) s.tslot[e] = K.tab_i32[e];
  for (int e = tid; e < 13 * N + NE; e += kThreads) s.tmem[e] = K.tab_u16[e];
  float *wl = (float *)(smem_raw + make_corr_layout(M, N, NP).wl);
  float *wW = wl, *wR = wl + 4 * (M + 1) * (M + 1), *wIn = wR + 4 * (M + 1);
  for (int e = tid; e < 4 * (M + 1) * (M + 1); e += kThreads) wW[e] = K.wallWf[e];
  for (int e = tid; e < 4 * (M + 1); e += kThreads) {
    wR[e] = K.wallRf[e];
    wIn[e] = K.wallInf[e];
  }
  __syncthreads();
  const int *lines = s.tslot + K.ln_off;
  const int *iqs = s.tslot + K.iq_off;  // heat-flux indices [3][4], then idx(e_i + e_j)
  const int i12 = iqs[12 + 1];
  const int ncell = L.ncell;
  const long long total = (long long)steps * 4 * ncell;
  const float Cf = (float)K.C;
  float *dsm = corr_defect(smem_raw, M, N, NP);
  const int VS = corr_vstride(M, NP);  // row stride of the transform vectors in VA / VB
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
    // ---- the data that stays fixed during the launch (the cell's defect row; each stencil
    //      cell's frozen coefficients and FP32 state) is copied asynchronously at once; then
    //      per stencil slot (warp w takes slot w, warp 0 also slot 8) the warp waits until the
    //      cell's correction words carry the version of the serial order (the newest for a
    //      neighbour that sweep Dk visits earlier, the previous one otherwise) and copies them.
    //      A satisfied cell cannot change again before this update is published, so rows that
    //      are ready early load while the last dependency is pending.
    for (int q = tid; q < NP / 4; q += kThreads) cp_async16(dsm + 4 * q, L.d32 + (size_t)c * NP + 4 * q);
    {
      const int warp = tid >> 5, lane = tid & 31;
      const int si = (k == 0 || k == 3) ? 1 : -1, sj = (k == 0 || k == 1) ? 1 : -1;
      for (int sl = warp; sl < 9; sl += kThreads / 32) {
        const int di = c_nb_di[sl], dj = c_nb_dj[sl];
        const int ii = i + di, jj = j + dj;
        const bool in = ii >= 0 && ii < L.nx && jj >= 0 && jj < L.ny && abs(di) + abs(dj) <= K.reach;
        if (lane == 0) {
          s.iarr[I_EX + sl] = in ? 1 : 0;
          if (sl >= 1 && sl <= 4) s.iarr[I_WALL + sl - 1] = in ? 0 : 1;  // face f = slot f + 1
        }
        if (!in) continue;  // warp-uniform
        const int cc = c + dj * L.nx + di;
        float *row = cstencil(s, sl, NP), *srow = ss + sl * NP;
        if (lane < 2) cp_async16(row + 4 * lane, L.aux32 + (size_t)cc * 8 + 4 * lane);
        for (int q = lane; q < NP / 4; q += 32) cp_async16(srow + 4 * q, L.s32 + (size_t)cc * NP + 4 * q);
        const bool before = (si * di < 0) || (di == 0 && sj * dj < 0);
        const int need = (sl != 0 && before) ? v : v - 1;
        if (!ll_row(K, s.eidx, L.et + (size_t)cc * NP, row + 8, need, lane) && lane == 0) s.iarr[I_ABW] = 1;
      }
    }
    cp_async_wait_all();
    __syncthreads();
    if (s.iarr[I_ABW]) break;
    const float *ac = s.cst, *ec = s.cst + 8;  // own frozen coefficients, own correction
    // ---- face states of the correction, slots as in the FP64 operator: 2f / 2f+1 = face f's
    //      left / right state (E, W, N, S), or 2f = the cell in the wall basis at a wall.  One
    //      thread per element (e < 4: the frozen params, which give the face bases; else the
    //      correction coefficient eidx[e - 4]) forms that element of every face state.
    {
      unsigned ex = 0;
#pragma unroll
      for (int sl = 0; sl < 9; ++sl) ex |= (s.iarr[I_EX + sl] ? 1u : 0u) << sl;
      const bool wallW = s.iarr[I_WALL + 1], wallS = s.iarr[I_WALL + 3];
      const bool slopes = K.reach == 2 && K.slope != 0;
      // coefficient lanes fill whole warps; the four params go to the next warp, so that no
      // warp runs both kinds
      const int ncw = (NE + 31) & ~31;
      for (int qe = tid; qe < ncw + 4; qe += kThreads) {
        if (qe < ncw && qe >= NE) continue;
        const int e = qe < ncw ? 4 + qe : qe - ncw;
        const bool par = e < 4;
        const int o = par ? e : s.eidx[e - 4];
        const int col = par ? e : 8 + o;
        float q[9], w[9];
#pragma unroll
        for (int sl = 0; sl < 9; ++sl) {
          q[sl] = ((ex >> sl) & 1u) ? cstencil(s, sl, NP)[col] : 0.0f;
          w[sl] = (!par && ((ex >> sl) & 1u)) ? ss[sl * NP + o] : 0.0f;
        }
        // slope items: 0 C along x, 1 C along y, 2 E, 3 W, 4 N, 5 S (cell X, lower Xm, upper Xp)
        constexpr int itx[6] = {0, 0, 1, 2, 3, 4}, itm[6] = {2, 4, 0, 6, 0, 8}, itp[6] = {1, 3, 5, 0, 7, 0};
#pragma unroll
        for (int it = 0; it < 6; ++it) {
          const int X = itx[it], Xm = itm[it], Xp = itp[it];
          if (!((ex >> X) & 1u)) continue;
          const bool on = slopes && ((ex >> Xm) & 1u) && ((ex >> Xp) & 1u);
          const float q0 = q[X];
          float hs = 0.0f;
          if (on) {
            // reconstruction factors of the item's cell: 1, 1, 1/4 on a uniform grid
            float rm = 1.0f, rp = 1.0f, ch = 0.25f;
            if (!L.uniform) {
              if (it == 1 || it >= 4) {
                const int r = j + c_nb_dj[X];
                rm = (float)L.rmy[r], rp = (float)L.rpy[r], ch = (float)L.chy[r];
              } else {
                const int cl = i + c_nb_di[X];
                rm = (float)L.rmx[cl], rp = (float)L.rpx[cl], ch = (float)L.chx[cl];
              }
            }
            const float qm = q[Xm], qp = q[Xp];
            if (par) {  // face basis: the reconstructed params of the state
              hs = L.uniform ? half_slope_f(K.slope, qm, q0, qp)
                             : (K.slope == 1 ? (qp - qm) * ch
                                             : half_slope_f(K.slope, q0 - (q0 - qm) * rm, q0, q0 + (qp - q0) * rp));
            } else if (K.slope == 1) {  // correction: the limited slope linearized with frozen weights
              hs = L.uniform ? 0.25f * (qp - qm) : (qp - qm) * ch;
            } else if (L.uniform) {
              const float a = w[X] - w[Xm], b = w[Xp] - w[X];
              const float den = fmaf(a, a, fmaf(b, b, 2e-12f));
              hs = __fdividef(0.5f * (fmaf(b, b, 1e-12f) * (q0 - qm) + fmaf(a, a, 1e-12f) * (qp - q0)), den);
            } else {
              const float a = (w[X] - w[Xm]) * rm, b = (w[Xp] - w[X]) * rp;
              const float den = fmaf(a, a, fmaf(b, b, 2e-12f));
              hs = __fdividef(0.5f * (fmaf(b, b, 1e-12f) * (q0 - qm) * rm + fmaf(a, a, 1e-12f) * (qp - q0) * rp), den);
            }
          }
          int v0, v1 = -1;
          float x0, x1 = 0.0f;
          switch (it) {
            case 0:
              v0 = 0; x0 = q0 + hs;
              if (wallW) { v1 = 2; x1 = q0; } else { v1 = 3; x1 = q0 - hs; }
              break;
            case 1:
              v0 = 4; x0 = q0 + hs;
              if (wallS) { v1 = 6; x1 = q0; } else { v1 = 7; x1 = q0 - hs; }
              break;
            case 2: v0 = 1; x0 = q0 - hs; break;
            case 3: v0 = 2; x0 = q0 + hs; break;
            case 4: v0 = 5; x0 = q0 - hs; break;
            default: v0 = 6; x0 = q0 + hs; break;
          }
          if (par) {
            s.vsrc[v0 * 4 + e] = x0;
            if (v1 >= 0) s.vsrc[v1 * 4 + e] = x1;
          } else {
            s.VA[v0 * VS + o] = x0;
            if (v1 >= 0) s.VA[v1 * VS + o] = x1;
          }
        }
      }
    }
    // destination bases: the cell, or the wall for a wall face's slot 2f
    if (tid >= 192 && tid < 224) {
      int vv = (tid - 192) >> 2, e = tid & 3, f = vv >> 1;
      if (s.iarr[I_WALL + f] && !(vv & 1)) {
        int w = c_face_wall[f];
        s.vdst[vv * 4 + e] = e < 3 ? (float)K.wall_u[w][e] : (float)K.wall_theta[w];
      } else {
        s.vdst[vv * 4 + e] = ac[e];
      }
    }
    if (tid == 224) {
      int na = 0;
      for (int f = 0; f < 4; ++f) {
        s.iarr[I_ACT + na++] = 2 * f;
        if (!s.iarr[I_WALL + f]) s.iarr[I_ACT + na++] = 2 * f + 1;
      }
      s.iarr[I_NACT] = na;
    }
    if (tid >= 228 && tid < 231 && K.model == 1) {
      int ii = tid - 228;
      const int *iq = iqs + 4 * ii;
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
    // batch 0: face states -> cell basis and the cell -> wall bases; batch 1 (cells with a
    // wall face): the wall fluxes -> cell basis.  One call site keeps one inlined copy.
    for (int batch = 0;; ++batch) {
      setup_coeffs(K, s);
      __syncthreads();
      if (M < kLineMax)
        transform_lines(K, s, lines, s.VA, s.VB, VS);
      else
        transform_batch(K, s, s.VA, s.VB);
      if (batch == 1) break;
      // ---- wall fluxes (linear in the face state)
      if (tid < 4 && s.iarr[I_WALL + tid]) {
        int w = c_face_wall[tid], ax = c_wall_axis[w];
        const float *a = s.VB + (2 * tid) * VS;
        const float *wr = wR + w * (M + 1);
        float rw = 0.0f;
        for (int m = 0; m <= M; ++m) rw = fmaf(wr[m], a[K.idx_axis[ax][m]], rw);
        s.sc[C_RHOW + tid] = rw;
      }
      __syncthreads();
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
        const float *a = s.VB + (2 * f) * VS;
        const float *Wm = wW + (size_t)w * (M + 1) * (M + 1) + p * (M + 1);
        const uint16_t *mem = s.tmem + ax * N;
        float g = 0.0f;
        for (int m = 0; m <= Lm; ++m) g = fmaf(a[mem[b0 + m]], Wm[m], g);
        if (deg == p) g = fmaf(s.sc[C_RHOW + f], wIn[w * (M + 1) + p], g);
        s.VA[(2 * f) * VS + o] = g;
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
      if (nw == 0) break;
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
          ee[ax] = fmaf(sg, s.VB[(2 * fc) * VS + o], ee[ax]);
        } else {
          float am = s.VB[(2 * fc) * VS + o], ap = s.VB[(2 * fc + 1) * VS + o];
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
    unsigned long long *Eo = L.et + (size_t)c * NP;
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
      // the tagged word publishes the value: no barrier or release store follows (the next
      // item's first barrier keeps this item's shared memory until every thread is done)
      st_relaxed_u64(Eo + o, tag_word(fmaf(dt, R - dsm[o], ec[o]), v));
    }
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
      s.VA[o] = L.F[(size_t)c * NP + o] + (double)word_value(L.et[(size_t)c * NP + o]);
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

// ------------------------------------------------------------------ learned field correction
// f <- Grad(f + increment) with the increment of the ten learned fields (rho, u1, u2, theta,
// s11, s12, s22, s33, q1, q2) d = U s y / 10 written into the cell's own Grad expansion:
// rho += d_rho; f_{e_i} += rho' d_u_i; every f_{2e_d} += rho' (3 d_theta + |d_u|^2) / 6 (the
// temperature of the new velocity); f_{e_i+e_j} += d_s_ij / (1 + delta_ij) with the trace of d_s
// removed; f_{3e_i} and f_{e_i+2e_d} += d_q_i / 5 (q_i = 2 f_{3e_i} + sum_d f_{e_i+2e_d}).
__global__ void __launch_bounds__(kThreads) field_correct_kernel(Consts K, LevelDev L, const float *y, const double *sdev,
                                                                 double U) {
  extern __shared__ __align__(16) char smem_raw[];
  Sm s = bind_smem_f64(smem_raw, K.M, K.N, K.NP);
  const int tid = threadIdx.x, N = K.N, NE = K.NE, NP = K.NP;
  for (int e = tid; e < 3 * NE + N; e += kThreads) s.tslot[e] = K.tab_i32[e];
  for (int e = tid; e < 13 * N + NE; e += kThreads) s.tmem[e] = K.tab_u16[e];
  __syncthreads();
  const int *iq = K.tab_i32 + K.iq_off, *is = iq + 12;  // heat-flux indices [3][4]; idx(e_i + e_j), i <= j
  const double fac = U * sdev[0] / 10.0;
  for (int c = blockIdx.x; c < L.ncell; c += gridDim.x) {
    const float *yc = y + (size_t)c * 10;
    double d[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) d[k] = fac * (double)yc[k];
    const double rho1 = L.F[(size_t)c * NP] + d[0];
    const double tr = (d[4] + d[6] + d[7]) * (1.0 / 3.0);
    const double iso = rho1 * (3.0 * d[3] + d[1] * d[1] + d[2] * d[2]) * (1.0 / 6.0);
    for (int q = tid; q < NE; q += kThreads) {
      const int o = s.eidx[q];
      double v = L.F[(size_t)c * NP + o];
      if (o == 0) v += d[0];
      if (o == K.idx_e[0]) v += rho1 * d[1];
      if (o == K.idx_e[1]) v += rho1 * d[2];
      if (o == K.idx_2e[0]) v += iso + 0.5 * (d[4] - tr);
      if (o == K.idx_2e[1]) v += iso + 0.5 * (d[6] - tr);
      if (o == K.idx_2e[2]) v += iso + 0.5 * (d[7] - tr);
      if (o == is[1]) v += d[5];
      for (int i = 0; i < 2; ++i)
        for (int m = 0; m < 3; ++m)
          if (o == iq[4 * i + 1 + m] && (m != i || o == iq[4 * i])) v += 0.2 * d[8 + i];
      s.VA[o] = v;
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
  cudaFuncSetAttribute(field_correct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
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

cudaError_t launch_field_correct(const Consts &K, const LevelDev &L, const float *y, const double *s_dev, double U,
                                 int grid, cudaStream_t st) {
  init_attrs_mixed();
  size_t sm = make_layout(K.M, K.N, K.NP).total;
  field_correct_kernel<<<grid, kThreads, sm, st>>>(K, L, y, s_dev, U);
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
