// Device machinery shared by the FP64 kernels (nrmg_kernels.cu) and the FP32 correction sweeps
// (nrmg_mixed.cu): shared-memory layout, index tables, memory-model helpers and the batched
// Hermite basis transform.
#pragma once
#include "nrmg_internal.h"

#include <math.h>

namespace nrmg {

#define VA_EPS2 1e-12  // van Albada smoothing constant (squared)

// ------------------------------------------------------------------ shared-memory layout
// cst: the cell's own state (params + coefficients).  VB doubles as the stencil buffer: the
// eight neighbour states are only read while the face states are built, before the first
// transform pass overwrites VB.
struct SLayout {
  size_t cst, VA, VB, vsrc, vdst, cf, sc, fact, ti32, vflag, iarr, tu16, total;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline size_t vb_doubles(int NP) {
  size_t a = (size_t)kNV * NP, b = (size_t)8 * (4 + NP);
  return a > b ? a : b;
}

constexpr int kScal = 128;  // doubles of per-cell scalars

__host__ __device__ inline SLayout make_layout(int M, int N, int NP) {
  const int NE = nmom_even(M);
  SLayout s;
  size_t o = 0;
  s.cst = o;   o = al16(o + sizeof(double) * (4 + NP));
  s.VA = o;    o = al16(o + sizeof(double) * kNV * NP);
  s.VB = o;    o = al16(o + sizeof(double) * vb_doubles(NP));
  s.vsrc = o;  o = al16(o + sizeof(double) * kNV * 4);
  s.vdst = o;  o = al16(o + sizeof(double) * kNV * 4);
  s.cf = o;    o = al16(o + sizeof(double) * kNV * 3 * (M + 1));
  s.sc = o;    o = al16(o + sizeof(double) * kScal);
  s.fact = o;  o = al16(o + sizeof(double) * N);
  s.ti32 = o;  o = al16(o + sizeof(int) * (3 * NE + N));
  s.vflag = o; o = al16(o + sizeof(int) * kNV * 3);
  s.iarr = o;  o = al16(o + sizeof(int) * 64);
  s.tu16 = o;  o = al16(o + sizeof(uint16_t) * (13 * N + NE));
  s.total = o;
  return s;
}


// Shared-memory working set of one cell update; T is the arithmetic type (double for the plain
// path, float for the FP32 correction sweeps).
template <typename T>
struct SmT {
  T *cst, *VA, *VB, *vsrc, *vdst, *cf, *sc;
  double *fact;
  int *tslot, *tshak, *vflag, *iarr;
  uint16_t *tmem, *tprev, *tnext, *tal, *tdeg, *eidx;
};
using Sm = SmT<double>;

// iarr slots
enum { I_ITEM = 0, I_NACT = 1, I_ACT = 2 /* ..2+kNV */, I_EX = 16 /* ..16+9 */, I_WALL = 28 /* ..28+4 */,
       I_BAD = 34, I_ABORT = 35, I_ABW = 36 /* a dependency wait of this item gave up */ };
// sc slots
enum { S_DT = 0, S_NU = 1, S_Q = 2 /* ..5 */, S_W = 8 /* ..8+12: w1,w2,w3 per face */, S_RHOW = 20 /* ..24 */,
       S_NEWP = 24 /* ..28 */, S_PH = 32 /* ..36 */, S_NORM = 40, S_TPN = 42, S_RED = 44 /* ..44+8 warps */,
       S_TPOW = 64 /* ..64+kMaxM+1: theta^-k */,
       // ES-BGK equilibrium factors: (B_dd/2)^m/m! for d = 1..3, m <= kMaxM/2, and B_12^k/k!
       S_ESG = 82 /* ..82+3*(kMaxM/2+1) */, S_ESH = 110 /* ..110+kMaxM+1 */ };
static_assert(S_ESH + kMaxM + 1 <= kScal && S_TPOW + kMaxM + 1 <= S_ESG, "per-cell scalar slots overlap");

constexpr uint16_t kNone = 0xFFFF;

__device__ inline Sm bind_smem(char *base, int M, int N, int NP) {
  SLayout L = make_layout(M, N, NP);
  Sm s;
  s.cst = (double *)(base + L.cst);
  s.VA = (double *)(base + L.VA);
  s.VB = (double *)(base + L.VB);
  s.vsrc = (double *)(base + L.vsrc);
  s.vdst = (double *)(base + L.vdst);
  s.cf = (double *)(base + L.cf);
  s.sc = (double *)(base + L.sc);
  s.fact = (double *)(base + L.fact);
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

// state of stencil slot sl (0 = the cell, 1..8 = neighbours E, W, N, S, EE, WW, NN, SS)
__device__ inline double *stencil(const Sm &s, int sl, int NP) {
  return sl == 0 ? s.cst : s.VB + (size_t)(sl - 1) * (4 + NP);
}

__device__ inline void load_tables(const Consts &K, Sm &s) {
  const int N = K.N;
  for (int e = threadIdx.x; e < 3 * K.NE + N; e += kThreads) s.tslot[e] = K.tab_i32[e];
  for (int e = threadIdx.x; e < 13 * N + K.NE; e += kThreads) s.tmem[e] = K.tab_u16[e];
  for (int e = threadIdx.x; e < N; e += kThreads) s.fact[e] = K.tab_f64[e];
}

// ------------------------------------------------------------------ memory-model helpers
__device__ inline int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ inline void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ inline unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ inline int ld_volatile(const int *p) { return *(const volatile int *)p; }

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per wait

__device__ inline void raise_status(const Consts &K, int code, bool abort_all) {
  atomicCAS(K.status, 0, code);
  if (abort_all) atomicExch(K.abort_flag, 1);
}

// ------------------------------------------------------------------ batched basis transform
// 1/(k+1), k = 0..kMaxM+1, so the coefficient recurrence needs no division
static __constant__ double c_inv[kMaxM + 2] = {1.0,       1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,  1.0 / 6,
                                        1.0 / 7,   1.0 / 8,  1.0 / 9,  1.0 / 10, 1.0 / 11, 1.0 / 12,
                                        1.0 / 13,  1.0 / 14, 1.0 / 15, 1.0 / 16, 1.0 / 17, 1.0 / 18};

// Coefficients of exp(-a z - b z^2) = sum_k c_k z^k for every active vector and direction:
// c_0 = 1, c_1 = -a, (k+1) c_{k+1} = -a c_k - 2 b c_{k-1}, with a = w~_d - w_d, b = (t~ - t)/2.
// The factors -a/(k+1) and -2b/(k+1) do not depend on the chain, so each step costs one
// dependent FMA.  Flags: bit 0 the direction is the identity, bit 1 a = 0 (odd c_k vanish
// exactly).
static __constant__ float c_invf[kMaxM + 2] = {1.0f,       1.0f / 2,  1.0f / 3,  1.0f / 4,  1.0f / 5,
                                               1.0f / 6,   1.0f / 7,  1.0f / 8,  1.0f / 9,  1.0f / 10,
                                               1.0f / 11,  1.0f / 12, 1.0f / 13, 1.0f / 14, 1.0f / 15,
                                               1.0f / 16,  1.0f / 17, 1.0f / 18};
__device__ inline double cinv(double, int k) { return c_inv[k]; }
__device__ inline float cinv(float, int k) { return c_invf[k]; }

template <typename T>
__device__ inline void setup_coeffs(const Consts &K, SmT<T> &s) {
  const int M = K.M, na = s.iarr[I_NACT];
  for (int t = threadIdx.x; t < na * 3; t += kThreads) {
    int v = s.iarr[I_ACT + t / 3], d = t % 3;
    T a = s.vdst[v * 4 + d] - s.vsrc[v * 4 + d];
    T b = T(0.5) * (s.vdst[v * 4 + 3] - s.vsrc[v * 4 + 3]);
    T *c = s.cf + (v * 3 + d) * (M + 1);
    T cm = T(1), ck = -a;
    c[0] = cm;
    c[1] = ck;
#pragma unroll
    for (int k = 1; k < kMaxM; ++k) {
      if (k >= M) break;
      T u = (T(-2) * b * cinv(T(0), k)) * cm;
      T cn = fma(-a * cinv(T(0), k), ck, u);
      c[k + 1] = cn;
      cm = ck;
      ck = cn;
    }
    s.vflag[v * 3 + d] = ((a == T(0) && b == T(0)) ? 1 : 0) | (a == T(0) ? 2 : 0);
  }
}

// one output coefficient of a directional pass: sum_k c_k x_{alpha - k e_d} over the
// non-vanishing k, split over two accumulators so that two FMA chains run side by side
template <typename T>
__device__ inline T transform_one(const T *x, const T *c, const uint16_t *mem, int o, int s0, int p, int fl) {
  T a0 = x[o];
  if (fl & 1) return a0;
  const int st = (fl & 2) ? 2 : 1;
  if (p < 2 * st) {  // at most one term: one chain, no closing add (the FP64 pipe is the bound)
    if (st <= p) a0 = fma(c[st], x[mem[s0 - st]], a0);
    return a0;
  }
  T a1 = T(0);
  int k = st;
  for (; k + st <= p; k += 2 * st) {
    a0 = fma(c[k], x[mem[s0 - k]], a0);
    a1 = fma(c[k + st], x[mem[s0 - k - st]], a1);
  }
  if (k <= p) a0 = fma(c[k], x[mem[s0 - k]], a0);
  return a0 + a1;
}

// g = prod_d exp(-a_d S_d - b S_d^2) f for the active vectors: passes X->Y, Y->X, X->Y.
// Output alpha of direction d sums c_k f_{alpha - k e_d}, k = 0..alpha_d; the index line of
// alpha along d is stored contiguously in tmem (s0 = position of alpha itself).  Only the
// outputs with even alpha_3 are formed: for planar states (u_3 = 0, odd alpha_3 coefficients
// zero) the others stay exactly zero, and directions 1, 2 and the even-k direction-3 series
// map even alpha_3 onto even alpha_3.  Each thread forms two outputs at a time (independent
// FMA chains: dependent FP64 latency, not throughput, limits a single cell update).
// Barrier over the first n threads of the CTA (named barrier 1, n a multiple of 32): every
// warp below n / 32 must reach it, and no other warp may.
__device__ __forceinline__ void bar_first(int n) { asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory"); }

// nbar < kThreads: the passes synchronize only the first nbar threads (the caller guarantees
// that threads from nbar on have no output, i.e. na * NE <= nbar).
template <typename T>
__device__ inline void transform_batch(const Consts &K, SmT<T> &s, T *X, T *Y, int nbar = kThreads) {
  const int N = K.N, NE = K.NE, NP = K.NP, M = K.M, na = s.iarr[I_NACT];
  const int tot = na * NE;
  for (int d = 0; d < 3; ++d) {
    const T *in = (d == 1) ? Y : X;
    T *out = (d == 1) ? X : Y;
    const int *slot = s.tslot + d * NE;
    const uint16_t *mem = s.tmem + d * N;
    for (int q = threadIdx.x; q < tot; q += 2 * kThreads) {
      const int q2 = q + kThreads;
      int vi = q / NE, r = q - vi * NE;
      int v = s.iarr[I_ACT + vi];
      int pk = slot[r];
      int o = pk & 2047;
      T y0 = transform_one(in + v * NP, s.cf + (v * 3 + d) * (M + 1), mem, o, (pk >> 11) & 2047, pk >> 22,
                           s.vflag[v * 3 + d]);
      T y1 = T(0);
      int v2 = 0, o2 = 0;
      if (q2 < tot) {
        int vi2 = q2 / NE, r2 = q2 - vi2 * NE;
        v2 = s.iarr[I_ACT + vi2];
        int pk2 = slot[r2];
        o2 = pk2 & 2047;
        y1 = transform_one(in + v2 * NP, s.cf + (v2 * 3 + d) * (M + 1), mem, o2, (pk2 >> 11) & 2047, pk2 >> 22,
                           s.vflag[v2 * 3 + d]);
      }
      out[v * NP + o] = y0;
      if (q2 < tot) out[v2 * NP + o2] = y1;
    }
    if (nbar == kThreads)
      __syncthreads();
    else
      bar_first(nbar);
  }
}

// rho, u, theta of g in a general basis p (eq. rho-u-theta with the moments of H_alpha);
// planar: f_{e_3} = 0.
__device__ inline void macros(const Consts &K, const double *p, const double *g, double *out) {
  double rho = g[0], f2 = 0.0, fe2 = 0.0, fe[3];
  const double ir = 1.0 / rho;
  for (int d = 0; d < 3; ++d) {
    fe[d] = d < 2 ? g[K.idx_e[d]] : 0.0;
    f2 += g[K.idx_2e[d]];
    fe2 += fe[d] * fe[d];
  }
  out[0] = rho;
  for (int d = 0; d < 3; ++d) out[1 + d] = fma(fe[d], ir, p[d]);
  out[4] = fma(fma(2.0, f2, -fe2 * ir), ir * (1.0 / 3.0), p[3]);
}

// Half of the limited slope times the cell width, q_face = q0 +- hs (eq. moments-recon with the
// slope of the central difference, or of the van Albada average (b^2+e)a + (a^2+e)b over
// a^2 + b^2 + 2e = (a+b)(ab+e) / (a^2+b^2+2e), a = q0 - qm, b = qp - q0).
// 1/x for x >= 2e-12 (normal, finite): the hardware reciprocal estimate refined by two
// Newton-Raphson steps y <- y + y (1 - x y) (each step squares the relative error).
__device__ inline double rcp_nr(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

__device__ inline double half_slope(int slope, double qm, double q0, double qp) {
  if (slope == 1) return 0.25 * (qp - qm);
  double a = q0 - qm, b = qp - q0;
  return 0.5 * ((a + b) * fma(a, b, VA_EPS2)) * rcp_nr(fma(a, a, fma(b, b, 2.0 * VA_EPS2)));
}

// The same on a non-uniform grid, with the factors of the cell's column or row: the central
// slope times h/2 is (qp - qm) ch; the van Albada average takes the one-sided differences
// scaled to the cell's width, a = (q0 - qm) rm, b = (qp - q0) rp.
__device__ inline double half_slope_nu(int slope, double qm, double q0, double qp, double rm, double rp,
                                       double ch) {
  if (slope == 1) return (qp - qm) * ch;
  double a = (q0 - qm) * rm, b = (qp - q0) * rp;
  return 0.5 * ((a + b) * fma(a, b, VA_EPS2)) * rcp_nr(fma(a, a, fma(b, b, 2.0 * VA_EPS2)));
}

// inverse widths of column i and row j, area of cell (i, j)
__device__ inline double inv_hx(const LevelDev &L, int i) { return L.uniform ? L.idx : L.ihx[i]; }
__device__ inline double inv_hy(const LevelDev &L, int j) { return L.uniform ? L.idy : L.ihy[j]; }
__device__ inline double cell_area(const LevelDev &L, int i, int j) {
  return L.uniform ? L.dx * L.dy : L.hx[i] * L.hy[j];
}

// stencil slots: 0 C, 1 E, 2 W, 3 N, 4 S, 5 EE, 6 WW, 7 NN, 8 SS
static __constant__ int c_nb_di[9] = {0, 1, -1, 0, 0, 2, -2, 0, 0};
static __constant__ int c_nb_dj[9] = {0, 0, 0, 1, -1, 0, 0, 2, -2};
// slope items: cell X with its lower / upper neighbours along the item's axis
static __constant__ int c_it_x[6] = {0, 0, 1, 2, 3, 4};
static __constant__ int c_it_m[6] = {2, 4, 0, 6, 0, 8};
static __constant__ int c_it_p[6] = {1, 3, 5, 0, 7, 0};
static __constant__ int c_face_wall[4] = {1, 3, 2, 0};  // wall index behind face E, W, N, S
static __constant__ int c_face_nb[4] = {1, 2, 3, 4};    // stencil slot across face E, W, N, S
static __constant__ int c_wall_axis[4] = {1, 0, 1, 0};

__device__ inline double block_sum(double v, double *red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < kThreads / 32; ++k) t += red[k];
  return t;  // valid in thread 0
}

}  // namespace nrmg
