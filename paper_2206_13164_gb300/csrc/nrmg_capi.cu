// Host side of the C ABI declared in include/nrmg.h: argument checks, index tables, the
// layout of the caller's workspace, and the FAS cycle of Algorithm 2 issued as kernel launches
// on the caller's stream.
#include "nrmg.h"
#include "nrmg_internal.h"
#include "nrmg_net.h"

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

using namespace nrmg;

namespace {

// ------------------------------------------------------------------ index tables
struct Tables {
  int M = 0, N = 0, NE = 0;
  std::vector<int> al;           // [N][3]
  std::vector<int32_t> i32;      // tslot[3][NE], tshak[N], iq[12], is[6], index lines (tab_i32_size)
  std::vector<uint16_t> u16;     // tmem[3N], tprev[3N], tnext[3N], tal[3N], tdeg[N], eidx[NE]
  std::vector<double> fact;      // [N]
  int idx_axis[2][kMaxM + 1];
  int idx_e[3], idx_2e[3];
};

int nmom(int M) { return (M + 1) * (M + 2) * (M + 3) / 6; }

// entries of tab_i32: tslot[3][NE], tshak[N], iq[12], is[6], then the line tables
int tab_i32_size(int M) { return 3 * nmom_even(M) + nmom(M) + 18 + nlines_total(M); }

void build_tables(int M, Tables &T) {
  T.M = M;
  T.N = nmom(M);
  const int N = T.N;
  T.al.resize(3 * N);
  std::vector<int> cube((M + 1) * (M + 1) * (M + 1), -1);
  auto cidx = [&](int a, int b, int c) -> int {
    if (a < 0 || b < 0 || c < 0 || a + b + c > M) return -1;
    return cube[(a * (M + 1) + b) * (M + 1) + c];
  };
  int k = 0;
  for (int deg = 0; deg <= M; ++deg)
    for (int a1 = deg; a1 >= 0; --a1)
      for (int a2 = deg - a1; a2 >= 0; --a2) {
        int a3 = deg - a1 - a2;
        T.al[3 * k] = a1;
        T.al[3 * k + 1] = a2;
        T.al[3 * k + 2] = a3;
        cube[(a1 * (M + 1) + a2) * (M + 1) + a3] = k++;
      }
  // the outputs formed by the kernels: multi-indices with even alpha_3 (planar states)
  std::vector<int> even;
  for (int o = 0; o < N; ++o)
    if (T.al[3 * o + 2] % 2 == 0) even.push_back(o);
  const int NE = (int)even.size();
  T.NE = NE;
  T.i32.assign(tab_i32_size(M), -1);
  T.u16.assign(13 * N + NE, 0xFFFF);
  T.fact.resize(N);
  for (int q = 0; q < NE; ++q) T.u16[13 * N + q] = (uint16_t)even[q];
  for (int d = 0; d < 3; ++d) {
    // index lines along d: all alpha sharing alpha with alpha_d = 0, stored by ascending alpha_d
    std::vector<int> s0(N, -1);
    int pos = 0;
    for (int o = 0; o < N; ++o) {
      const int *a = &T.al[3 * o];
      if (a[d] != 0) continue;
      for (int m = 0;; ++m) {
        int t[3] = {a[0], a[1], a[2]};
        t[d] = m;
        int q = cidx(t[0], t[1], t[2]);
        if (q < 0) break;
        T.u16[d * N + pos] = (uint16_t)q;
        s0[q] = pos++;
      }
    }
    // outputs (even alpha_3) sorted by line position (alpha_d) descending: a warp runs
    // equal-length loops
    std::vector<int> ord(even);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return T.al[3 * x + d] > T.al[3 * y + d]; });
    for (int r = 0; r < NE; ++r) {
      int o = ord[r];
      T.i32[d * NE + r] = o | (s0[o] << 11) | (T.al[3 * o + d] << 22);
    }
    for (int o = 0; o < N; ++o) {
      int t[3] = {T.al[3 * o], T.al[3 * o + 1], T.al[3 * o + 2]};
      t[d] -= 1;
      int pm = cidx(t[0], t[1], t[2]);
      t[d] += 2;
      int pp = cidx(t[0], t[1], t[2]);
      T.u16[3 * N + d * N + o] = pm < 0 ? 0xFFFF : (uint16_t)pm;
      T.u16[6 * N + d * N + o] = pp < 0 ? 0xFFFF : (uint16_t)pp;
      T.u16[9 * N + d * N + o] = (uint16_t)T.al[3 * o + d];
    }
  }
  // line tables: per direction, (start in that direction's tmem segment) | (length << 11),
  // longest first (a warp's lanes then run chains of similar length)
  {
    int off = 3 * NE + N + 18;
    for (int d = 0; d < 3; ++d) {
      std::vector<std::pair<int, int>> ln;  // (length, start)
      int pos = 0;
      for (int o = 0; o < N; ++o) {
        const int *a = &T.al[3 * o];
        if (a[d] != 0) continue;
        const int L = M + 1 - (a[0] + a[1] + a[2]);
        if (d == 2 || a[2] % 2 == 0) ln.push_back({L, pos});
        pos += L;
      }
      std::stable_sort(ln.begin(), ln.end(), [](const std::pair<int, int> &x, const std::pair<int, int> &y) {
        return x.first > y.first;
      });
      for (size_t q = 0; q < ln.size(); ++q) T.i32[off + q] = ln[q].second | (ln[q].first << 11);
      off += (int)ln.size();
    }
  }
  for (int o = 0; o < N; ++o) {
    const int *a = &T.al[3 * o];
    T.u16[12 * N + o] = (uint16_t)(a[0] + a[1] + a[2]);
    double f = 1.0;
    for (int d = 0; d < 3; ++d)
      for (int q = 2; q <= a[d]; ++q) f *= q;
    T.fact[o] = f;
    // Shakhov target: alpha = 3 e_i, or e_i + 2 e_d with d != i
    int sh = -1;
    for (int i = 0; i < 3; ++i) {
      if (a[i] == 3 && a[0] + a[1] + a[2] == 3) sh = i;
      for (int d = 0; d < 3; ++d)
        if (d != i && a[i] == 1 && a[d] == 2 && a[0] + a[1] + a[2] == 3) sh = i;
    }
    T.i32[3 * NE + o] = sh;
  }
  // heat-flux indices iq[i] = {3e_i, 2e_0+e_i, 2e_1+e_i, 2e_2+e_i} and sigma indices e_i+e_j
  for (int i = 0; i < 3; ++i) {
    int e3[3] = {0, 0, 0};
    e3[i] = 3;
    T.i32[3 * NE + N + 4 * i] = cidx(e3[0], e3[1], e3[2]);
    for (int d = 0; d < 3; ++d) {
      int t[3] = {0, 0, 0};
      t[d] += 2;
      t[i] += 1;
      T.i32[3 * NE + N + 4 * i + 1 + d] = cidx(t[0], t[1], t[2]);
    }
  }
  int q = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      int t[3] = {0, 0, 0};
      t[i] += 1;
      t[j] += 1;
      T.i32[3 * NE + N + 12 + q++] = cidx(t[0], t[1], t[2]);
    }
  for (int ax = 0; ax < 2; ++ax)
    for (int m = 0; m <= kMaxM; ++m) {
      int t[3] = {0, 0, 0};
      t[ax] = m;
      T.idx_axis[ax][m] = m <= M ? cidx(t[0], t[1], t[2]) : -1;
    }
  for (int d = 0; d < 3; ++d) {
    int t[3] = {0, 0, 0};
    t[d] = 1;
    T.idx_e[d] = cidx(t[0], t[1], t[2]);
    t[d] = 2;
    T.idx_2e[d] = cidx(t[0], t[1], t[2]);
  }
}

// Largest root of He_n: largest eigenvalue of the Jacobi matrix (zero diagonal, off-diagonal
// sqrt(k)), by bisection on the Sturm sequence count.
double hermite_largest_root(int n) {
  if (n <= 1) return 0.0;
  auto count_below = [&](double x) {  // number of eigenvalues < x
    int cnt = 0;
    double q = -x;
    if (q < 0) ++cnt;
    for (int k = 1; k < n; ++k) {
      double qq = (q == 0.0) ? 1e-300 : q;
      q = -x - k / qq;
      if (q < 0) ++cnt;
    }
    return cnt;
  };
  double lo = 0.0, hi = 2.0 * sqrt((double)n) + 1.0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (count_below(mid) < n)
      lo = mid;
    else
      hi = mid;
  }
  return 0.5 * (lo + hi);
}

// Half-range moments J^s_{k,m} = int_{s v > 0} v He_k(v) He_m(v) phi(v) dv, via the
// linearization He_k He_m = sum_j C(k,j) C(m,j) j! He_{k+m-2j}, v He_n = He_{n+1} + n He_{n-1}
// and int_0^inf He_n phi = He_{n-1}(0) phi(0) (n >= 1), 1/2 (n = 0).  Long double limits the
// cancellation of the alternating sum.
void halfrange_table(int K, int s, std::vector<double> &J) {
  typedef long double ld;
  const ld pi = 3.141592653589793238462643383279502884L;
  std::vector<ld> he0(2 * K + 4, 0.0L), A(2 * K + 4, 0.0L);
  he0[0] = 1.0L;
  he0[1] = 0.0L;
  for (int n = 1; n + 1 < (int)he0.size(); ++n) he0[n + 1] = -(ld)n * he0[n - 1];
  A[0] = 0.5L;
  for (int n = 1; n < (int)A.size(); ++n) A[n] = he0[n - 1] / sqrtl(2.0L * pi);
  auto vint = [&](int n) -> ld { return A[n + 1] + (n >= 1 ? (ld)n * A[n - 1] : 0.0L); };  // int_0^inf v He_n phi
  J.assign((K + 1) * (K + 1), 0.0);
  for (int k = 0; k <= K; ++k)
    for (int m = 0; m <= K; ++m) {
      ld acc = 0.0L, ck = 1.0L, cm = 1.0L, jf = 1.0L;
      for (int j = 0; j <= std::min(k, m); ++j) {
        if (j > 0) {
          ck = ck * (ld)(k - j + 1) / (ld)j;
          cm = cm * (ld)(m - j + 1) / (ld)j;
          jf *= (ld)j;
        }
        acc += ck * cm * jf * vint(k + m - 2 * j);
      }
      // J^- = (-1)^{k+m+1} J^+ (reflection v -> -v)
      ld sg = ((k + m + 1) % 2 == 0) ? 1.0L : -1.0L;
      J[k * (K + 1) + m] = (double)(s > 0 ? acc : sg * acc);
    }
}

const int kWallAxis[4] = {1, 0, 1, 0};
const int kWallSign[4] = {-1, +1, +1, -1};

// Wall matrices of the half-range Maxwell flux: W[k][m] = theta^((k-m+1)/2)/k!
// (J^s_{k,m} + (1-chi)(-1)^m J^{-s}_{k,m}); rho_w = sum_m R[m] a_{m e_n} with
// R[m] = s sqrt(2 pi) theta^(-m/2) J^s_{0,m}; incoming Maxwellian In[k] = chi theta^((k+1)/2)/k! J^{-s}_{k,0}.
void wall_tables(int M, const nrmg_wall *walls, std::vector<double> &W, std::vector<double> &R,
                 std::vector<double> &In) {
  const int K1 = M + 1;
  W.assign(4 * K1 * K1, 0.0);
  R.assign(4 * K1, 0.0);
  In.assign(4 * K1, 0.0);
  for (int w = 0; w < 4; ++w) {
    int s = kWallSign[w];
    double th = walls[w].theta, chi = walls[w].chi;
    std::vector<double> Js, Jm;
    halfrange_table(M, s, Js);
    halfrange_table(M, -s, Jm);
    double kf = 1.0;
    for (int k = 0; k <= M; ++k) {
      if (k > 0) kf *= k;
      for (int m = 0; m <= M; ++m) {
        double sg = (m % 2 == 0) ? 1.0 : -1.0;
        W[(w * K1 + k) * K1 + m] = pow(th, 0.5 * (k - m + 1)) / kf * (Js[k * K1 + m] + (1.0 - chi) * sg * Jm[k * K1 + m]);
      }
      In[w * K1 + k] = chi * pow(th, 0.5 * (k + 1)) / kf * Jm[k * K1 + 0];
    }
    for (int m = 0; m <= M; ++m) R[w * K1 + m] = s * sqrt(2.0 * M_PI) * pow(th, -0.5 * m) * Js[0 * K1 + m];
  }
}

// ------------------------------------------------------------------ sweep schedules
// Cells of sweep Dk (k = 0..3 for D1..D4) by anti-diagonal, then by i.
void sweep_order(int nx, int ny, int k, int *o) {
  int n = 0;
  bool idesc = (k == 1 || k == 2), jdesc = (k == 2 || k == 3);
  for (int dg = 0; dg <= nx + ny - 2; ++dg)
    for (int a = 0; a < nx; ++a) {
      int b = dg - a;
      if (b < 0 || b >= ny) continue;
      int i = idesc ? nx - 1 - a : a, j = jdesc ? ny - 1 - b : b;
      o[n++] = j * nx + i;
    }
}

// Order of the items (s, k, c) of FS^steps by their earliest start in the dependency graph of
// the exact sweep (longest path from the initial state, each update counted as one unit): the
// update of cell c to version v = 4s + k + 1 depends on c's version v - 1 and on each cross
// neighbour within `reach` at version v (visited before c by sweep Dk) or v - 1 (after).  The
// order is topological, so CTAs taking items in this order never wait on an item not yet
// taken, and items of consecutive sweeps and steps interleave as early as the serial order
// allows.
void asap_schedule_keys(int nx, int ny, int reach, int steps, std::vector<std::pair<int, int>> &keys);

void asap_schedule(int nx, int ny, int reach, int steps, std::vector<int> &queue) {
  std::vector<std::pair<int, int>> keys;
  asap_schedule_keys(nx, ny, reach, steps, keys);
  queue.resize(keys.size());
  for (size_t q = 0; q < keys.size(); ++q) queue[q] = keys[q].second;
}

// (start time, item) of every item of FS^steps, sorted by start time (see asap_schedule)
void asap_schedule_keys(int nx, int ny, int reach, int steps, std::vector<std::pair<int, int>> &keys) {
  const int nc = nx * ny, V = 4 * steps;
  std::vector<int> tv((size_t)(V + 1) * nc, 0);
  std::vector<int> ord(nc);
  keys.clear();
  keys.reserve((size_t)V * nc);
  const int di[8] = {1, -1, 0, 0, 2, -2, 0, 0}, dj[8] = {0, 0, 1, -1, 0, 0, 2, -2};
  const int nnb = reach == 2 ? 8 : 4;
  for (int st = 0; st < steps; ++st)
    for (int k = 0; k < 4; ++k) {
      sweep_order(nx, ny, k, ord.data());
      const int v = 4 * st + k + 1;
      const int si = (k == 0 || k == 3) ? 1 : -1, sj = (k == 0 || k == 1) ? 1 : -1;
      for (int n = 0; n < nc; ++n) {
        const int c = ord[n], i = c % nx, j = c / nx;
        int tmax = tv[(size_t)(v - 1) * nc + c];
        for (int q = 0; q < nnb; ++q) {
          int ii = i + di[q], jj = j + dj[q];
          if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) continue;
          bool before = (si * di[q] < 0) || (di[q] == 0 && sj * dj[q] < 0);
          int w = before ? v : v - 1;
          tmax = std::max(tmax, tv[(size_t)w * nc + jj * nx + ii]);
        }
        tv[(size_t)v * nc + c] = tmax + 1;
        keys.push_back({tmax + 1, (st * 4 + k) * nc + c});
      }
    }
  std::stable_sort(keys.begin(), keys.end(),
                   [](const std::pair<int, int> &a, const std::pair<int, int> &b) { return a.first < b.first; });
}

// ------------------------------------------------------------------ workspace layout
struct Carver {
  size_t off = 0;
  char *base = nullptr;
  template <typename T>
  T *take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T *p = base ? (T *)(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

int pad4(int n) { return (n + 3) & ~3; }
constexpr int kPartials = 8192;

}  // namespace

struct nrmg_ctx {
  nrmg_grid grid;
  int M, N, NP, levels;
  double Kn;
  nrmg_wall walls[4];
  nrmg_collision coll;
  nrmg_opts opts;
  cudaStream_t stream;
  int nsm;
  int occ[4];
  int occ_corr;
  int fs_ctas_per_sm;  // persistent CTAs per SM of the sweep launches (0: the occupancy)
  int cluster_cells;   // FP64 sweeps of levels with at most this many cells use two-CTA clusters
  int cluster_cap[2];  // two-CTA clusters that fit with 1 and 2 CTAs per SM (0: unavailable)
  Consts K;
  LevelDev lev[kMaxLev];
  struct {
    int steps;
    int *queue;
  } sched[kMaxLev][4];
  int nsched[kMaxLev];
  double *partials, *dscal;   // reduction scratch, device scalars
  int *dstatus;
  double *hpin;               // pinned host scalars
  int *hpin_i;
  double m0, res0;
  int have_res0;
  int ref_fixed;              // res0 set by nrmg_set_reference: solves keep it
  int mixed_off;              // precision 1: FP64 smoothing for the rest of this solve (stall)
  int mixed_stalled;          // the last nrmg_solve switched to FP64 smoothing
  long long launches;
  // event timing of FS launches
  int profiling;
  std::vector<cudaEvent_t> ev;
  std::vector<long long> ev_upd;   // cell updates of each timed launch
  std::vector<int> ev_hasr;
  std::vector<int> ev_level;
  std::vector<int> ev_prec;   // 0 FP64 sweep, 1 FP32 correction sweep
  size_t ev_used;
  // event timing of residual launches (all modes)
  std::vector<cudaEvent_t> rev;
  std::vector<long long> rev_cells;
  std::vector<int> rev_hasr;
  size_t rev_used;
  char err[256];
};

namespace {

// step counts with a precomputed schedule: 1 and the FS counts of Algorithm 2 on that level
std::vector<int> sched_steps(int level, const nrmg_opts *o) {
  std::vector<int> v = {1};
  auto add = [&](int x) {
    if (x > 0 && std::find(v.begin(), v.end(), x) == v.end()) v.push_back(x);
  };
  if (level == 0) add(o->s3);
  add(o->s1);
  add(o->s2);
  return v;
}

void layout(const nrmg_grid *g, int M, const nrmg_opts *opts, Carver &cv, nrmg_ctx *ctx) {
  const int N = nmom(M), NP = pad4(N), NE = nmom_even(M);
  // tables
  int32_t *ti = cv.take<int32_t>(tab_i32_size(M));
  uint16_t *tu = cv.take<uint16_t>(13 * N + NE);
  double *tf = cv.take<double>(N);
  double *wW = cv.take<double>(4 * (M + 1) * (M + 1));
  double *wR = cv.take<double>(4 * (M + 1));
  double *wI = cv.take<double>(4 * (M + 1));
  float *wWf = cv.take<float>(4 * (M + 1) * (M + 1));
  float *wRf = cv.take<float>(4 * (M + 1));
  float *wIf = cv.take<float>(4 * (M + 1));
  int *ctl = cv.take<int>(64);  // status, abort, queue
  double *part = cv.take<double>(kPartials);
  double *scal = cv.take<double>(64);
  LevelDev lv[kMaxLev];
  for (int l = g->levels - 1; l >= 0; --l) {
    int sh = g->levels - 1 - l;
    LevelDev &L = lv[l];
    L.nx = g->nx >> sh;
    L.ny = g->ny >> sh;
    L.ncell = L.nx * L.ny;
    L.dx = g->lx / L.nx;
    L.dy = g->ly / L.ny;
    L.idx = 1.0 / L.dx;
    L.idy = 1.0 / L.dy;
    size_t nc = L.ncell;
    L.P = cv.take<double>(nc * 4);
    L.F = cv.take<double>(nc * NP);
    L.rP = cv.take<double>(nc * 4);
    L.rF = cv.take<double>(nc * NP);
    L.bP = cv.take<double>(nc * 4);
    L.bF = cv.take<double>(nc * NP);
    L.D = cv.take<double>(nc * NP);
    L.tp = cv.take<double>(nc);
    L.ver = cv.take<int>(nc);
    L.order = cv.take<int>(4 * nc);
    L.has_r = 0;
    // geometry of a non-uniform grid (filled by nrmg_set_spacing): per column hx, 1/hx, rm, rp,
    // ch, then the same per row
    double *geo = cv.take<double>(5 * (size_t)(L.nx + L.ny));
    L.uniform = 1;
    L.hx = geo;
    L.ihx = geo + L.nx;
    L.rmx = geo + 2 * L.nx;
    L.rpx = geo + 3 * L.nx;
    L.chx = geo + 4 * L.nx;
    L.hy = geo + 5 * L.nx;
    L.ihy = L.hy + L.ny;
    L.rmy = L.hy + 2 * L.ny;
    L.rpy = L.hy + 3 * L.ny;
    L.chy = L.hy + 4 * L.ny;
    if (opts->precision == 1) {
      L.et = cv.take<unsigned long long>(nc * NP);
      L.d32 = cv.take<float>(nc * NP);
      L.aux32 = cv.take<float>(nc * 8);
      L.s32 = cv.take<float>(nc * NP);
    } else {
      L.et = nullptr;
      L.d32 = L.aux32 = L.s32 = nullptr;
    }
    int ns = 0;
    for (int steps : sched_steps(l, opts)) {
      int *q = cv.take<int>((size_t)steps * 4 * nc);
      if (ctx) {
        ctx->sched[l][ns].steps = steps;
        ctx->sched[l][ns].queue = q;
      }
      ++ns;
    }
    if (ctx) ctx->nsched[l] = ns;
  }
  if (ctx) {
    ctx->K.tab_i32 = ti;
    ctx->K.tab_u16 = tu;
    ctx->K.tab_f64 = tf;
    ctx->K.wallW = wW;
    ctx->K.wallRho = wR;
    ctx->K.wallIn = wI;
    ctx->K.wallWf = wWf;
    ctx->K.wallRf = wRf;
    ctx->K.wallInf = wIf;
    ctx->K.status = ctl;
    ctx->K.abort_flag = ctl + 1;
    ctx->K.queue = ctl + 2;
    ctx->dstatus = ctl;
    ctx->partials = part;
    ctx->dscal = scal;
    for (int l = 0; l < g->levels; ++l) ctx->lev[l] = lv[l];
  }
}

bool grid_ok(const nrmg_grid *g) {
  if (!g || g->levels < 1 || g->levels > kMaxLev || g->nx < 1 || g->ny < 1) return false;
  if (!(g->lx > 0.0) || !(g->ly > 0.0)) return false;
  int sh = g->levels - 1;
  if ((g->nx >> sh) < 1 || (g->ny >> sh) < 1) return false;
  if (((g->nx >> sh) << sh) != g->nx || ((g->ny >> sh) << sh) != g->ny) return false;
  if ((long long)g->nx * g->ny > (1LL << 28)) return false;
  return true;
}

bool opts_ok(const nrmg_opts *o) {
  if (!o) return false;
  if (o->order != 1 && o->order != 2) return false;
  if (o->slope < 0 || o->slope > 2) return false;
  if (!(o->dtnu >= 0.0)) return false;
  if (!(o->cfl > 0.0) || o->s1 < 0 || o->s2 < 0 || o->s3 < 0 || o->gamma < 1 || o->gamma > 2) return false;
  if (o->precision != 0 && o->precision != 1) return false;
  return true;
}

nrmg_status set_err(nrmg_ctx *c, nrmg_status s, const char *msg) {
  if (c) snprintf(c->err, sizeof(c->err), "%s", msg);
  return s;
}

nrmg_status cuda_check(nrmg_ctx *c, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return NRMG_OK;
  if (c) snprintf(c->err, sizeof(c->err), "%s: %s", what, cudaGetErrorString(e));
  return NRMG_ERR_CUDA;
}

#define CK(expr)                                            \
  do {                                                      \
    nrmg_status _s = cuda_check(ctx, (expr), #expr);        \
    if (_s != NRMG_OK) return _s;                           \
  } while (0)

// FP64 sweeps of levels up to 128 x 128 cells split each update over a two-CTA cluster by
// default, with one cluster CTA per SM up to 64 x 64 cells and two per SM above.  Measured
// on GB300 (256 x 256, M = 10 V-cycle, single CTAs at 2 per SM): the 8^2 ... 64^2 levels'
// sweeps run 1.4x faster on 76 clusters, the 128^2 level's 1.3x faster on 152; the 256^2
// level loses on either (it already has enough single-CTA updates in flight).
constexpr int kClusterCellsDefault = 128 * 128;
constexpr int kClusterSparseCells = 64 * 64;

int grid_for(nrmg_ctx *ctx, int which, long long work) {
  int per_sm = std::max(1, ctx->occ[which]);
  if (which == 0 && ctx->fs_ctas_per_sm > 0) per_sm = std::min(per_sm, ctx->fs_ctas_per_sm);
  long long g = (long long)ctx->nsm * per_sm;
  if (work < g) g = work;
  if (g > kPartials) g = kPartials;
  return (int)std::max(1LL, g);
}

// device status -> host, then clear it
nrmg_status sync_status(nrmg_ctx *ctx) {
  CK(cudaMemcpyAsync(ctx->hpin_i, ctx->dstatus, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  int st = ctx->hpin_i[0];
  if (st != 0) {
    CK(cudaMemsetAsync(ctx->dstatus, 0, 2 * sizeof(int), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    snprintf(ctx->err, sizeof(ctx->err), "device reported status %d", st);
    return (nrmg_status)st;
  }
  return NRMG_OK;
}

nrmg_status smooth(nrmg_ctx *ctx, int level, int steps) {
  if (steps <= 0) return NRMG_OK;
  LevelDev &L = ctx->lev[level];
  CK(cudaMemsetAsync(L.ver, 0, sizeof(int) * L.ncell, ctx->stream));
  CK(cudaMemsetAsync(ctx->K.queue, 0, sizeof(int), ctx->stream));
  int g = grid_for(ctx, 0, (long long)steps * 4 * L.ncell);
  const int *queue = nullptr;
  for (int q = 0; q < ctx->nsched[level]; ++q)
    if (ctx->sched[level][q].steps == steps) queue = ctx->sched[level][q].queue;
  bool timed = ctx->profiling && ctx->ev_used + 2 <= ctx->ev.size();
  if (timed) CK(cudaEventRecord(ctx->ev[ctx->ev_used], ctx->stream));
  if (ctx->cluster_cap[0] > 0 && L.ncell <= ctx->cluster_cells) {
    // one cluster CTA per SM while the level's wavefront is short; two per SM (twice the
    // clusters) once it is longer than the clusters one per SM could serve
    const int dense = (L.ncell > kClusterSparseCells && ctx->cluster_cap[1] > 0) ? 1 : 0;
    const long long nc = std::min<long long>(ctx->cluster_cap[dense], (long long)steps * 4 * L.ncell);
    CK(launch_fs_cluster(ctx->K, L, steps, queue, (int)nc, dense + 1, ctx->stream));
  } else {
    CK(launch_fs(ctx->K, L, steps, queue, g, ctx->stream));
  }
  if (timed) {
    CK(cudaEventRecord(ctx->ev[ctx->ev_used + 1], ctx->stream));
    ctx->ev_upd[ctx->ev_used / 2] = (long long)steps * 4 * L.ncell;
    ctx->ev_hasr[ctx->ev_used / 2] = L.has_r;
    ctx->ev_level[ctx->ev_used / 2] = level;
    ctx->ev_prec[ctx->ev_used / 2] = 0;
    ctx->ev_used += 2;
  }
  ctx->launches += 1;
  return NRMG_OK;
}

// residual of a level: mode kResOut (R - r, dense stride out_stride, norm partials),
// kResDefect, kResCoarseRhs
nrmg_status residual(nrmg_ctx *ctx, int level, int mode, double *out, int out_stride, int *grid_out) {
  LevelDev L = ctx->lev[level];
  if (mode == kResCoarseRhs) L.has_r = 0;
  int g = grid_for(ctx, 1, L.ncell);
  bool timed = ctx->profiling && ctx->rev_used + 2 <= ctx->rev.size();
  if (timed) CK(cudaEventRecord(ctx->rev[ctx->rev_used], ctx->stream));
  CK(launch_residual(ctx->K, L, mode, out, out_stride, ctx->partials, g, ctx->stream));
  if (timed) {
    CK(cudaEventRecord(ctx->rev[ctx->rev_used + 1], ctx->stream));
    ctx->rev_cells[ctx->rev_used / 2] = L.ncell;
    ctx->rev_hasr[ctx->rev_used / 2] = L.has_r;
    ctx->rev_used += 2;
  }
  ctx->launches += 1;
  if (grid_out) *grid_out = g;
  return NRMG_OK;
}

// write_defect: the same residual evaluation also leaves L.D = r - R(f) (the mixed smoother's
// defect of this state)
nrmg_status norm_of(nrmg_ctx *ctx, int level, double *out_dev_R, double *norm_host, bool write_defect = false) {
  int g = 0;
  nrmg_status s = residual(ctx, level, write_defect ? kResDefectNorm : kResOut, out_dev_R, ctx->N, &g);
  if (s != NRMG_OK) return s;
  CK(launch_reduce_norm(ctx->partials, g, 1.0 / (ctx->grid.lx * ctx->grid.ly), ctx->dscal, ctx->stream));
  ctx->launches += 1;
  if (norm_host) {
    CK(cudaMemcpyAsync(ctx->hpin, ctx->dscal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    nrmg_status st = sync_status(ctx);
    if (st != NRMG_OK) return st;
    *norm_host = ctx->hpin[0];
  }
  return NRMG_OK;
}

nrmg_status two_grid_setup(nrmg_ctx *ctx, int lf) {
  nrmg_status s = residual(ctx, lf, kResDefect, nullptr, 0, nullptr);
  if (s != NRMG_OK) return s;
  LevelDev &Lc = ctx->lev[lf - 1];
  int g = grid_for(ctx, 2, Lc.ncell);
  CK(launch_restrict(ctx->K, ctx->lev[lf], Lc, g, ctx->stream));
  ctx->launches += 1;
  // the restricted defect is the coarse state's defect r_H - R_H(f_H): kept for the mixed
  // smoother's first coarse smoothing (it has no other use on a coarse level)
  if (ctx->opts.precision == 1)
    CK(cudaMemcpyAsync(Lc.D, Lc.rF, sizeof(double) * ctx->NP * Lc.ncell, cudaMemcpyDeviceToDevice, ctx->stream));
  s = residual(ctx, lf - 1, kResCoarseRhs, nullptr, 0, nullptr);
  if (s != NRMG_OK) return s;
  ctx->lev[lf - 1].has_r = 1;
  return NRMG_OK;
}

nrmg_status two_grid_update(nrmg_ctx *ctx, int lf) {
  int g = grid_for(ctx, 3, ctx->lev[lf].ncell);
  CK(launch_prolong(ctx->K, ctx->lev[lf], ctx->lev[lf - 1], g, ctx->stream));
  ctx->launches += 1;
  return NRMG_OK;
}

// Mixed-precision smoothing of level `level`: FP64 defect d = r - R(f), `steps` FP32 sweeps of
// the linearized correction equation L e = d (same cell order as Algorithm 1), then
// f <- Grad(f + e) in FP64.
// defect_ready: L.D already holds r - R(f) of the current state (the restricted defect of a
// level that two_grid_setup has just formed).
nrmg_status smooth_mixed(nrmg_ctx *ctx, int level, int steps, bool defect_ready = false) {
  if (steps <= 0) return NRMG_OK;
  LevelDev &L = ctx->lev[level];
  nrmg_status s;
  if (!defect_ready && (s = residual(ctx, level, kResDefect, nullptr, 0, nullptr)) != NRMG_OK) return s;
  CK(launch_mixed_prep(ctx->K, L, ctx->stream));  // also sets every correction word to version 0
  CK(cudaMemsetAsync(ctx->K.queue, 0, sizeof(int), ctx->stream));
  const int *queue = nullptr;
  for (int q = 0; q < ctx->nsched[level]; ++q)
    if (ctx->sched[level][q].steps == steps) queue = ctx->sched[level][q].queue;
  int per_sm = std::max(1, ctx->occ_corr);
  if (ctx->fs_ctas_per_sm > 0) per_sm = std::min(per_sm, ctx->fs_ctas_per_sm);
  long long g = (long long)ctx->nsm * per_sm;
  g = std::min<long long>(g, (long long)steps * 4 * L.ncell);
  bool timed = ctx->profiling && ctx->ev_used + 2 <= ctx->ev.size();
  if (timed) CK(cudaEventRecord(ctx->ev[ctx->ev_used], ctx->stream));
  CK(launch_fs_corr(ctx->K, L, steps, queue, (int)std::max(1LL, g), ctx->stream));
  if (timed) {
    CK(cudaEventRecord(ctx->ev[ctx->ev_used + 1], ctx->stream));
    ctx->ev_upd[ctx->ev_used / 2] = (long long)steps * 4 * L.ncell;
    ctx->ev_hasr[ctx->ev_used / 2] = L.has_r;
    ctx->ev_level[ctx->ev_used / 2] = level;
    ctx->ev_prec[ctx->ev_used / 2] = 1;
    ctx->ev_used += 2;
  }
  CK(launch_mixed_update(ctx->K, L, grid_for(ctx, 3, L.ncell), ctx->stream));
  ctx->launches += 3;
  return NRMG_OK;
}

nrmg_status smooth_level(nrmg_ctx *ctx, int level, int steps, bool defect_ready = false) {
  if (ctx->opts.precision == 1 && !ctx->mixed_off && level > 0) return smooth_mixed(ctx, level, steps, defect_ready);
  return smooth(ctx, level, steps);
}

// Algorithm 2 on level k
// first_visit: the coarse level has just been formed by two_grid_setup, so its defect r - R(f)
// is the restricted defect that two_grid_setup left in L.D (the mixed smoother then skips its
// own defect evaluation).
nrmg_status nmg(nrmg_ctx *ctx, int k, bool first_visit = false) {
  const nrmg_opts &o = ctx->opts;
  nrmg_status s;
  if (k == 0) return smooth(ctx, 0, o.s3);
  if ((s = smooth_level(ctx, k, o.s1, first_visit)) != NRMG_OK) return s;
  if ((s = two_grid_setup(ctx, k)) != NRMG_OK) return s;
  for (int g = 0; g < o.gamma; ++g)
    if ((s = nmg(ctx, k - 1, g == 0)) != NRMG_OK) return s;
  if ((s = two_grid_update(ctx, k)) != NRMG_OK) return s;
  return smooth_level(ctx, k, o.s2);
}

nrmg_status mass_correct(nrmg_ctx *ctx) {
  LevelDev &L = ctx->lev[ctx->levels - 1];
  int g = (int)std::min<long long>(std::max(1, (L.ncell + kThreads - 1) / kThreads), 1024);
  CK(launch_mass(ctx->K, L, ctx->partials, g, ctx->dscal + 2, ctx->m0, true, ctx->stream));
  ctx->launches += 3;
  return NRMG_OK;
}

nrmg_status set_maxwellian(nrmg_ctx *ctx) {
  int nmax = 0;
  for (int l = 0; l < ctx->levels; ++l) nmax = std::max(nmax, ctx->lev[l].ncell);
  std::vector<double> ones(nmax, 1.0);
  for (int l = 0; l < ctx->levels; ++l) {
    LevelDev &L = ctx->lev[l];
    CK(cudaMemsetAsync(L.P, 0, sizeof(double) * 4 * L.ncell, ctx->stream));
    CK(cudaMemsetAsync(L.F, 0, sizeof(double) * ctx->NP * L.ncell, ctx->stream));
    CK(cudaMemsetAsync(L.rP, 0, sizeof(double) * 4 * L.ncell, ctx->stream));
    CK(cudaMemsetAsync(L.rF, 0, sizeof(double) * ctx->NP * L.ncell, ctx->stream));
    CK(cudaMemsetAsync(L.D, 0, sizeof(double) * ctx->NP * L.ncell, ctx->stream));
    CK(cudaMemsetAsync(L.bP, 0, sizeof(double) * 4 * L.ncell, ctx->stream));
    CK(cudaMemsetAsync(L.bF, 0, sizeof(double) * ctx->NP * L.ncell, ctx->stream));
    CK(cudaMemcpy2DAsync(L.F, sizeof(double) * ctx->NP, ones.data(), sizeof(double), sizeof(double), L.ncell,
                         cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpy2DAsync(L.P + 3, sizeof(double) * 4, ones.data(), sizeof(double), sizeof(double), L.ncell,
                         cudaMemcpyHostToDevice, ctx->stream));
    CK(launch_tpow(ctx->K, L, ctx->stream));
    L.has_r = 0;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->m0 = ctx->grid.lx * ctx->grid.ly;
  ctx->have_res0 = 0;
  ctx->ref_fixed = 0;
  return NRMG_OK;
}

}  // namespace

extern "C" {

size_t nrmg_workspace_bytes(const nrmg_grid *grid, int M, const nrmg_opts *opts) {
  if (!grid_ok(grid) || M < 3 || M > kMaxM || !opts_ok(opts)) return 0;
  Carver cv;
  layout(grid, M, opts, cv, nullptr);
  return cv.off + 256;
}

nrmg_status nrmg_create(const nrmg_grid *grid, int M, double Kn, const nrmg_wall walls[4],
                        const nrmg_collision *coll, const nrmg_opts *opts, void *dev_workspace, size_t ws_bytes,
                        void *cuda_stream, nrmg_ctx **out) {
  if (!out) return NRMG_ERR_ARG;
  *out = nullptr;
  if (!grid_ok(grid) || M < 3 || M > kMaxM || !(Kn > 0.0) || !walls || !coll || !opts_ok(opts) || !dev_workspace)
    return NRMG_ERR_ARG;
  if (coll->model != NRMG_BGK && coll->model != NRMG_SHAKHOV && coll->model != NRMG_ESBGK) return NRMG_ERR_ARG;
  if (!(coll->beta > 0.0) || !(coll->Pr > 0.0) || !isfinite(coll->omega)) return NRMG_ERR_ARG;
  for (int w = 0; w < 4; ++w) {
    if (!(walls[w].theta > 0.0) || walls[w].chi < 0.0 || walls[w].chi > 1.0) return NRMG_ERR_ARG;
    if (walls[w].u[kWallAxis[w]] != 0.0 || walls[w].u[2] != 0.0) return NRMG_ERR_ARG;
  }
  if (((uintptr_t)dev_workspace & 255) != 0) return NRMG_ERR_ARG;
  if (ws_bytes < nrmg_workspace_bytes(grid, M, opts)) return NRMG_ERR_OOM;

  nrmg_ctx *ctx = new nrmg_ctx();
  memset(ctx->err, 0, sizeof(ctx->err));
  ctx->grid = *grid;
  ctx->M = M;
  ctx->N = nmom(M);
  ctx->NP = pad4(ctx->N);
  ctx->levels = grid->levels;
  ctx->Kn = Kn;
  memcpy(ctx->walls, walls, sizeof(nrmg_wall) * 4);
  ctx->coll = *coll;
  ctx->opts = *opts;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->launches = 0;
  ctx->profiling = 0;
  ctx->ev_used = 0;
  Carver cv;
  cv.base = (char *)dev_workspace;
  layout(grid, M, opts, cv, ctx);

  int dev = 0;
  nrmg_status s;
  if ((s = cuda_check(ctx, cudaGetDevice(&dev), "cudaGetDevice")) != NRMG_OK) goto fail;
  if ((s = cuda_check(ctx, cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, dev),
                      "cudaDeviceGetAttribute")) != NRMG_OK)
    goto fail;
  if ((s = cuda_check(ctx, cudaMallocHost((void **)&ctx->hpin, 64 * sizeof(double)), "cudaMallocHost")) != NRMG_OK)
    goto fail;
  ctx->hpin_i = (int *)(ctx->hpin + 32);
  {
    Consts &K = ctx->K;
    K.M = M;
    K.N = ctx->N;
    K.NP = ctx->NP;
    K.NE = nmom_even(M);
    K.iq_off = 3 * K.NE + K.N;
    K.ln_off = K.iq_off + 18;
    for (int d = 0; d < 3; ++d) K.nl[d] = nlines(M, d);
    K.reach = (opts->order == 2 && opts->slope != 0) ? 2 : 1;
    K.slope = opts->order == 2 ? opts->slope : 0;
    K.model = coll->model;
    K.Kn = Kn;
    K.Pr = coll->Pr;
    K.omega = coll->omega;
    K.beta = coll->beta;
    K.cfl = opts->cfl;
    K.dtnu = opts->dtnu;
    K.nu0 = coll->beta * sqrt(M_PI / 2.0) / Kn;
    K.C = hermite_largest_root(M + 1);
    K.lx = grid->lx;
    K.ly = grid->ly;
    for (int w = 0; w < 4; ++w) {
      for (int d = 0; d < 3; ++d) K.wall_u[w][d] = walls[w].u[d];
      K.wall_theta[w] = walls[w].theta;
    }
    Tables T;
    build_tables(M, T);
    memcpy(K.idx_axis, T.idx_axis, sizeof(T.idx_axis));
    memcpy(K.idx_e, T.idx_e, sizeof(T.idx_e));
    memcpy(K.idx_2e, T.idx_2e, sizeof(T.idx_2e));
    std::vector<double> W, R, In;
    wall_tables(M, walls, W, R, In);
    cudaStream_t st = ctx->stream;
#define CKF(expr)                                                   \
  if ((s = cuda_check(ctx, (expr), #expr)) != NRMG_OK) goto fail;
    CKF(cudaMemcpyAsync((void *)K.tab_i32, T.i32.data(), T.i32.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CKF(cudaMemcpyAsync((void *)K.tab_u16, T.u16.data(), T.u16.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, st));
    CKF(cudaMemcpyAsync((void *)K.tab_f64, T.fact.data(), T.fact.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CKF(cudaMemcpyAsync((void *)K.wallW, W.data(), W.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CKF(cudaMemcpyAsync((void *)K.wallRho, R.data(), R.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CKF(cudaMemcpyAsync((void *)K.wallIn, In.data(), In.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    {
      std::vector<float> Wf(W.begin(), W.end()), Rf(R.begin(), R.end()), If(In.begin(), In.end());
      CKF(cudaMemcpyAsync((void *)K.wallWf, Wf.data(), Wf.size() * sizeof(float), cudaMemcpyHostToDevice, st));
      CKF(cudaMemcpyAsync((void *)K.wallRf, Rf.data(), Rf.size() * sizeof(float), cudaMemcpyHostToDevice, st));
      CKF(cudaMemcpyAsync((void *)K.wallInf, If.data(), If.size() * sizeof(float), cudaMemcpyHostToDevice, st));
      CKF(cudaStreamSynchronize(st));
    }
    CKF(cudaMemsetAsync(ctx->dstatus, 0, 64 * sizeof(int), st));
    // sweep orders: cells of Dk by anti-diagonal, then by i
    for (int l = 0; l < ctx->levels; ++l) {
      LevelDev &L = ctx->lev[l];
      std::vector<int> ord(4 * (size_t)L.ncell);
      for (int k = 0; k < 4; ++k) sweep_order(L.nx, L.ny, k, ord.data() + (size_t)k * L.ncell);
      CKF(cudaMemcpyAsync(L.order, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice, st));
      CKF(cudaStreamSynchronize(st));
      for (int q = 0; q < ctx->nsched[l]; ++q) {
        std::vector<int> queue;
        asap_schedule(L.nx, L.ny, K.reach, ctx->sched[l][q].steps, queue);
        CKF(cudaMemcpyAsync(ctx->sched[l][q].queue, queue.data(), queue.size() * sizeof(int),
                            cudaMemcpyHostToDevice, st));
        CKF(cudaStreamSynchronize(st));
      }
    }
    for (int w = 0; w < 4; ++w) ctx->occ[w] = occupancy_cell(M, ctx->NP, w);
    ctx->occ_corr = opts->precision == 1 ? occupancy_corr(M, ctx->NP) : 0;
    ctx->cluster_cap[0] = cluster_capacity(ctx->K, 1);
    ctx->cluster_cap[1] = cluster_capacity(ctx->K, 2);
    ctx->cluster_cells = kClusterCellsDefault;
    if (ctx->occ[0] < 1) {
      s = set_err(ctx, NRMG_ERR_ARG, "shared-memory footprint too large for this M");
      goto fail;
    }
#undef CKF
  }
  if ((s = set_maxwellian(ctx)) != NRMG_OK) goto fail;
  *out = ctx;
  return NRMG_OK;
fail:
  if (ctx->hpin) cudaFreeHost(ctx->hpin);
  delete ctx;
  return s;
}

nrmg_status nrmg_destroy(nrmg_ctx *ctx) {
  if (!ctx) return NRMG_ERR_ARG;
  cudaStreamSynchronize(ctx->stream);
  for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  for (cudaEvent_t e : ctx->rev) cudaEventDestroy(e);
  if (ctx->hpin) cudaFreeHost(ctx->hpin);
  delete ctx;
  return NRMG_OK;
}

namespace {
// Tail of every state upload: admissibility check, theta^(1-omega) cache and, on the finest
// level, the reference mass and residual.
nrmg_status finish_state(nrmg_ctx *ctx, int level) {
  LevelDev &L = ctx->lev[level];
  CK(launch_check_state(ctx->K, L.P, L.F, ctx->NP, L.ncell, 0, ctx->stream));
  ctx->launches += 1;
  nrmg_status s = sync_status(ctx);
  if (s == NRMG_ERR_ARG) return set_err(ctx, s, "set_state: state is not planar (u3 or an odd-alpha3 coefficient is nonzero)");
  if (s != NRMG_OK) return set_err(ctx, s, "set_state: non-physical or non-finite state");
  CK(launch_tpow(ctx->K, L, ctx->stream));
  ctx->launches += 1;
  if (level == ctx->levels - 1) {
    // reference mass of the correction
    int g = (int)std::min<long long>(std::max(1, (L.ncell + kThreads - 1) / kThreads), 1024);
    CK(launch_mass(ctx->K, L, ctx->partials, g, ctx->dscal + 2, 0.0, false, ctx->stream));
    ctx->launches += 2;
    CK(cudaMemcpyAsync(ctx->hpin, ctx->dscal + 2, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->m0 = ctx->hpin[0];
    ctx->have_res0 = 0;
    ctx->ref_fixed = 0;
  }
  return NRMG_OK;
}
}  // namespace

nrmg_status nrmg_set_state(nrmg_ctx *ctx, int level, const double *P, const double *F) {
  if (!ctx || level < 0 || level >= ctx->levels || !P || !F) return NRMG_ERR_ARG;
  LevelDev &L = ctx->lev[level];
  CK(cudaMemcpyAsync(L.P, P, sizeof(double) * 4 * L.ncell, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(launch_pack(F, ctx->N, L.F, ctx->NP, L.ncell, ctx->N, ctx->stream));
  ctx->launches += 1;
  return finish_state(ctx, level);
}

nrmg_status nrmg_set_state_from_fields(nrmg_ctx *ctx, const double *fields) {
  if (!ctx || !fields) return NRMG_ERR_ARG;
  const int top = ctx->levels - 1;
  LevelDev &L = ctx->lev[top];
  CK(launch_grad13(fields, L.ncell, ctx->M, ctx->NP, L.P, L.F, ctx->stream));
  ctx->launches += 1;
  return finish_state(ctx, top);
}

nrmg_status nrmg_set_grid(nrmg_ctx *ctx, int ctas_per_sm) {
  if (!ctx || ctas_per_sm < 0 || ctas_per_sm > std::max(ctx->occ[0], ctx->occ_corr)) return NRMG_ERR_ARG;
  ctx->fs_ctas_per_sm = ctas_per_sm;
  return NRMG_OK;
}

namespace {
// per-column (or row) geometry of one level: widths, inverses and reconstruction factors, in
// the order of the workspace block (h, 1/h, rm, rp, ch)
void spacing_factors(const std::vector<double> &h, std::vector<double> &out) {
  const size_t n = h.size();
  out.assign(5 * n, 0.0);
  for (size_t i = 0; i < n; ++i) {
    out[i] = h[i];
    out[n + i] = 1.0 / h[i];
    // wall-adjacent cells take no slope along this axis: their factors are never read
    const double hm = i > 0 ? 0.5 * (h[i - 1] + h[i]) : h[i];
    const double hp = i + 1 < n ? 0.5 * (h[i] + h[i + 1]) : h[i];
    out[2 * n + i] = h[i] / hm;
    out[3 * n + i] = h[i] / hp;
    out[4 * n + i] = 0.5 * h[i] / (hm + hp);
  }
}
}  // namespace

nrmg_status nrmg_set_spacing(nrmg_ctx *ctx, const double *host_hx, const double *host_hy) {
  if (!ctx || !host_hx || !host_hy) return NRMG_ERR_ARG;
  const int top = ctx->levels - 1;
  std::vector<double> hx(host_hx, host_hx + ctx->grid.nx), hy(host_hy, host_hy + ctx->grid.ny);
  double sx = 0.0, sy = 0.0;
  for (double h : hx) {
    if (!(h > 0.0) || !isfinite(h)) return set_err(ctx, NRMG_ERR_ARG, "set_spacing: widths must be positive");
    sx += h;
  }
  for (double h : hy) {
    if (!(h > 0.0) || !isfinite(h)) return set_err(ctx, NRMG_ERR_ARG, "set_spacing: heights must be positive");
    sy += h;
  }
  if (fabs(sx - ctx->grid.lx) > 1e-12 * ctx->grid.lx || fabs(sy - ctx->grid.ly) > 1e-12 * ctx->grid.ly)
    return set_err(ctx, NRMG_ERR_ARG, "set_spacing: widths must add up to lx and ly");
  std::vector<double> gx, gy;
  for (int l = top; l >= 0; --l) {
    LevelDev &L = ctx->lev[l];
    if (l < top) {  // a coarse cell merges two columns (rows) of the next finer level
      std::vector<double> cx(L.nx), cy(L.ny);
      for (int i = 0; i < L.nx; ++i) cx[i] = hx[2 * i] + hx[2 * i + 1];
      for (int j = 0; j < L.ny; ++j) cy[j] = hy[2 * j] + hy[2 * j + 1];
      hx.swap(cx);
      hy.swap(cy);
    }
    spacing_factors(hx, gx);
    spacing_factors(hy, gy);
    CK(cudaMemcpyAsync((void *)L.hx, gx.data(), sizeof(double) * gx.size(), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync((void *)L.hy, gy.data(), sizeof(double) * gy.size(), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));  // the host vectors are reused by the next level
    L.uniform = 0;
  }
  return set_maxwellian(ctx);
}

nrmg_status nrmg_set_cluster(nrmg_ctx *ctx, int max_cells) {
  if (!ctx || max_cells < 0) return NRMG_ERR_ARG;
  ctx->cluster_cells = max_cells;
  return NRMG_OK;
}

int nrmg_cluster_capacity(const nrmg_ctx *ctx) { return ctx ? ctx->cluster_cap[0] : 0; }

int nrmg_grid_limit(const nrmg_ctx *ctx) { return ctx ? std::max(1, std::max(ctx->occ[0], ctx->occ_corr)) : 0; }

nrmg_status nrmg_set_reference(nrmg_ctx *ctx, double mass, double res0) {
  if (!ctx || !(mass >= 0.0) || !(res0 >= 0.0) || !isfinite(mass) || !isfinite(res0)) return NRMG_ERR_ARG;
  if (mass > 0.0) ctx->m0 = mass;
  if (res0 > 0.0) {
    ctx->res0 = res0;
    ctx->have_res0 = 1;
    ctx->ref_fixed = 1;
  }
  return NRMG_OK;
}

nrmg_status nrmg_get_state(nrmg_ctx *ctx, int level, double *P, double *F) {
  if (!ctx || level < 0 || level >= ctx->levels) return NRMG_ERR_ARG;
  LevelDev &L = ctx->lev[level];
  if (P) CK(cudaMemcpyAsync(P, L.P, sizeof(double) * 4 * L.ncell, cudaMemcpyDeviceToDevice, ctx->stream));
  if (F) {
    CK(launch_pack(L.F, ctx->NP, F, ctx->N, L.ncell, ctx->N, ctx->stream));
    ctx->launches += 1;
  }
  return NRMG_OK;
}

nrmg_status nrmg_set_state_host(nrmg_ctx *ctx, int level, const double *host_P, const double *host_F) {
  if (!ctx || level < 0 || level >= ctx->levels || !host_P || !host_F) return NRMG_ERR_ARG;
  LevelDev &L = ctx->lev[level];
  // one copy per array; the coefficient rows land in their padded device rows directly
  CK(cudaMemcpyAsync(L.P, host_P, sizeof(double) * 4 * L.ncell, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpy2DAsync(L.F, sizeof(double) * ctx->NP, host_F, sizeof(double) * ctx->N, sizeof(double) * ctx->N,
                       L.ncell, cudaMemcpyHostToDevice, ctx->stream));
  return finish_state(ctx, level);
}

nrmg_status nrmg_get_state_host(nrmg_ctx *ctx, int level, double *host_P, double *host_F) {
  if (!ctx || level < 0 || level >= ctx->levels) return NRMG_ERR_ARG;
  LevelDev &L = ctx->lev[level];
  if (host_P) CK(cudaMemcpyAsync(host_P, L.P, sizeof(double) * 4 * L.ncell, cudaMemcpyDeviceToHost, ctx->stream));
  if (host_F)
    CK(cudaMemcpy2DAsync(host_F, sizeof(double) * ctx->N, L.F, sizeof(double) * ctx->NP, sizeof(double) * ctx->N,
                         L.ncell, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return NRMG_OK;
}

nrmg_status nrmg_set_rhs(nrmg_ctx *ctx, int level, const double *rP, const double *rF) {
  if (!ctx || level < 0 || level >= ctx->levels) return NRMG_ERR_ARG;
  LevelDev &L = ctx->lev[level];
  if (!rP || !rF) {
    L.has_r = 0;
    return NRMG_OK;
  }
  CK(cudaMemcpyAsync(L.rP, rP, sizeof(double) * 4 * L.ncell, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(launch_pack(rF, ctx->N, L.rF, ctx->NP, L.ncell, ctx->N, ctx->stream));
  CK(launch_check_state(ctx->K, L.rP, L.rF, ctx->NP, L.ncell, 1, ctx->stream));
  ctx->launches += 2;
  nrmg_status s = sync_status(ctx);
  if (s == NRMG_ERR_ARG) return set_err(ctx, s, "set_rhs: right-hand side is not planar");
  if (s != NRMG_OK) return set_err(ctx, s, "set_rhs: non-finite right-hand side or theta <= 0");
  L.has_r = 1;
  return NRMG_OK;
}

nrmg_status nrmg_smooth(nrmg_ctx *ctx, int level, int steps) {
  if (!ctx || level < 0 || level >= ctx->levels || steps < 0) return NRMG_ERR_ARG;
  return smooth(ctx, level, steps);
}

// One forward Euler step of `level` (eq. euler-scheme): R - r of the old state into the level's
// defect buffer, with the norm partials; when norm_host is given, its norm (synchronizes) and,
// if that is at or below stop_at, no update; else the global step and the update.
static nrmg_status euler_step(nrmg_ctx *ctx, int level, double stop_at, double *norm_host, bool *stopped) {
  LevelDev &L = ctx->lev[level];
  int g = 0;
  nrmg_status s = residual(ctx, level, kResOut, L.D, ctx->NP, &g);
  if (s != NRMG_OK) return s;
  if (stopped) *stopped = false;
  if (norm_host) {
    CK(launch_reduce_norm(ctx->partials, g, 1.0 / (ctx->grid.lx * ctx->grid.ly), ctx->dscal, ctx->stream));
    CK(cudaMemcpyAsync(ctx->hpin, ctx->dscal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if ((s = sync_status(ctx)) != NRMG_OK) return s;
    *norm_host = ctx->hpin[0];
    ctx->launches += 1;
    if (*norm_host <= stop_at) {
      if (stopped) *stopped = true;
      return NRMG_OK;
    }
  }
  CK(launch_euler(ctx->K, L, ctx->dscal + 8, grid_for(ctx, 3, L.ncell), ctx->stream));
  ctx->launches += 2;
  return NRMG_OK;
}

nrmg_status nrmg_euler(nrmg_ctx *ctx, int level, int steps) {
  if (!ctx || level < 0 || level >= ctx->levels || steps < 0) return NRMG_ERR_ARG;
  for (int n = 0; n < steps; ++n) {
    nrmg_status s = euler_step(ctx, level, 0.0, nullptr, nullptr);
    if (s != NRMG_OK) return s;
  }
  return NRMG_OK;
}

nrmg_status nrmg_euler_solve(nrmg_ctx *ctx, double tol, int max_steps, int *steps_out, double *rel_res_out) {
  if (!ctx || !(tol >= 0.0) || max_steps < 0) return NRMG_ERR_ARG;
  const int K = ctx->levels - 1;
  ctx->lev[K].has_r = 0;
  nrmg_status s;
  if (!ctx->ref_fixed) {
    if ((s = norm_of(ctx, K, nullptr, &ctx->res0)) != NRMG_OK) return s;
    ctx->have_res0 = 1;
  }
  const double ref = ctx->res0;
  double nrm = 0.0, rr = ref > 0.0 ? 1.0 : 0.0;
  int n = 0;
  for (;;) {
    bool stopped = false;
    const bool last = n >= max_steps;
    // at the step budget only the norm is wanted: stop_at = infinity skips the update
    if ((s = euler_step(ctx, K, last ? INFINITY : tol * ref, &nrm, &stopped)) != NRMG_OK) break;
    rr = ref > 0.0 ? nrm / ref : 0.0;
    if (stopped) break;
    ++n;
  }
  if (steps_out) *steps_out = n;
  if (rel_res_out) *rel_res_out = rr;
  if (s == NRMG_OK && rr > tol) s = NRMG_ERR_NOT_CONVERGED;
  return s;
}

nrmg_status nrmg_residual(nrmg_ctx *ctx, int level, double *dev_R_out, double *norm_out) {
  if (!ctx || level < 0 || level >= ctx->levels) return NRMG_ERR_ARG;
  if (norm_out) return norm_of(ctx, level, dev_R_out, norm_out);
  return residual(ctx, level, kResOut, dev_R_out, ctx->N, nullptr);
}

namespace {
// One cycle of the finest level, the mass correction and the norm.  defect_fresh: the finest
// level's D holds r - R(f) of the current state (the previous norm of this solve left it);
// write_defect: the closing norm leaves it for the next cycle.
nrmg_status fas_cycle(nrmg_ctx *ctx, double *rel_res_out, bool defect_fresh, bool write_defect) {
  const int K = ctx->levels - 1;
  nrmg_status s;
  ctx->lev[K].has_r = 0;
  if (!ctx->have_res0) {
    if ((s = norm_of(ctx, K, nullptr, &ctx->res0)) != NRMG_OK) return s;
    ctx->have_res0 = 1;
  }
  if ((s = nmg(ctx, K, defect_fresh)) != NRMG_OK) return s;
  if ((s = mass_correct(ctx)) != NRMG_OK) return s;
  double r = 0.0;
  if ((s = norm_of(ctx, K, nullptr, &r, write_defect)) != NRMG_OK) return s;
  if (rel_res_out) *rel_res_out = ctx->res0 > 0.0 ? r / ctx->res0 : 0.0;
  return NRMG_OK;
}
}  // namespace

nrmg_status nrmg_fas_cycle(nrmg_ctx *ctx, double *rel_res_out) {
  if (!ctx) return NRMG_ERR_ARG;
  return fas_cycle(ctx, rel_res_out, false, false);
}

// ------------------------------------------------------------------ learned coarse-level correction
namespace {
// Workspace of nrmg_fas_cycle_learned: coarse fields before and after the coarse cycles, fine
// fields after the plain update, network input and output, the saved finest state, the scale.
struct LearnWs {
  double *cb, *ca, *fine, *bP, *bF, *btp, *cP, *cF, *ctp, *s;
  float *x, *y;
};
size_t learned_ws(const nrmg_ctx *ctx, char *base, LearnWs *w) {
  const LevelDev &Lf = ctx->lev[ctx->levels - 1], &Lc = ctx->lev[ctx->levels - 2];
  Carver cv;
  cv.base = base;
  LearnWs t;
  t.cb = cv.take<double>((size_t)Lc.ncell * 14);
  t.ca = cv.take<double>((size_t)Lc.ncell * 14);
  t.fine = cv.take<double>((size_t)Lf.ncell * 14);
  t.x = cv.take<float>((size_t)Lf.ncell * NRMG_CORR_CIN);
  t.y = cv.take<float>((size_t)Lf.ncell * NRMG_LEARN_COUT);
  t.bP = cv.take<double>((size_t)Lf.ncell * 4);
  t.bF = cv.take<double>((size_t)Lf.ncell * ctx->NP);
  t.btp = cv.take<double>((size_t)Lf.ncell);
  t.cP = cv.take<double>((size_t)Lf.ncell * 4);
  t.cF = cv.take<double>((size_t)Lf.ncell * ctx->NP);
  t.ctp = cv.take<double>((size_t)Lf.ncell);
  t.s = cv.take<double>(8);
  if (w) *w = t;
  return cv.off;
}
}  // namespace

size_t nrmg_learned_cycle_workspace_bytes(const nrmg_ctx *ctx) {
  if (!ctx || ctx->levels < 2) return 0;
  const LevelDev &Lf = ctx->lev[ctx->levels - 1], &Lc = ctx->lev[ctx->levels - 2];
  if (Lc.nx * 2 != Lf.nx || Lc.ny * 2 != Lf.ny) return 0;
  return learned_ws(ctx, nullptr, nullptr) + 256;
}

// copy of the finest level's state (params, coefficients, theta^(1-omega)) between the level and
// a workspace slot
static nrmg_status copy_state(nrmg_ctx *ctx, double *dP, double *dF, double *dtp, const double *sP, const double *sF,
                              const double *stp) {
  const LevelDev &Lf = ctx->lev[ctx->levels - 1];
  CK(cudaMemcpyAsync(dP, sP, sizeof(double) * 4 * Lf.ncell, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemcpyAsync(dF, sF, sizeof(double) * ctx->NP * Lf.ncell, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemcpyAsync(dtp, stp, sizeof(double) * Lf.ncell, cudaMemcpyDeviceToDevice, ctx->stream));
  return NRMG_OK;
}

nrmg_status nrmg_fas_cycle_learned(nrmg_ctx *ctx, nrmg_net *net, const float *dev_y, int accept_rule, double Kn, double U,
                                   void *dev_ws, size_t ws_bytes, float *dev_x_out, double *dev_fine_out,
                                   double *scale_out, int *accepted_out, double *rel_res_out) {
  if (!ctx || !dev_ws || ((uintptr_t)dev_ws & 255) != 0 || !(Kn > 0.0) || !(U > 0.0)) return NRMG_ERR_ARG;
  if (accept_rule != NRMG_ACCEPT_UPDATE && accept_rule != NRMG_ACCEPT_SMOOTHED && accept_rule != NRMG_ACCEPT_ALWAYS) return NRMG_ERR_ARG;
  const size_t need = nrmg_learned_cycle_workspace_bytes(ctx);
  if (need == 0 || ws_bytes < need) return NRMG_ERR_ARG;
  const int K = ctx->levels - 1;
  LevelDev &Lf = ctx->lev[K], &Lc = ctx->lev[K - 1];
  if (net && !net_fits(net, NRMG_CORR_CIN, NRMG_LEARN_COUT, (long long)Lf.ncell, ctx->stream)) return NRMG_ERR_ARG;
  LearnWs w;
  learned_ws(ctx, (char *)dev_ws, &w);
  float *x = dev_x_out ? dev_x_out : w.x;
  double *fine = dev_fine_out ? dev_fine_out : w.fine;
  const nrmg_opts &o = ctx->opts;
  cudaStream_t st = ctx->stream;
  nrmg_status s;
  Lf.has_r = 0;
  if (!ctx->have_res0) {
    if ((s = norm_of(ctx, K, nullptr, &ctx->res0)) != NRMG_OK) return s;
    ctx->have_res0 = 1;
  }
  // Algorithm 2 on the finest level (as nmg), with the coarse change and the plain update open
  if ((s = smooth_level(ctx, K, o.s1)) != NRMG_OK) return s;
  if ((s = two_grid_setup(ctx, K)) != NRMG_OK) return s;
  CK(launch_fields(ctx->K, Lc, w.cb, st));
  for (int g = 0; g < o.gamma; ++g)
    if ((s = nmg(ctx, K - 1, g == 0)) != NRMG_OK) return s;
  CK(launch_fields(ctx->K, Lc, w.ca, st));
  if ((s = two_grid_update(ctx, K)) != NRMG_OK) return s;
  CK(launch_fields(ctx->K, Lf, fine, st));
  CK(launch_corr_inputs(w.cb, w.ca, Lc.ny, Lc.nx, fine, ctx->grid.lx, ctx->grid.ly, Kn, U, w.s, x, st));
  ctx->launches += 5;
  int accepted = 0;
  bool smoothed = false;  // the level already holds the post-smoothed winner
  if (net || dev_y) {
    const float *y = dev_y;
    if (net) {
      if ((s = nrmg_net_forward(net, x, 1, Lf.ny, Lf.nx, w.y)) != NRMG_OK) return s;
      y = w.y;
    }
    double r_plain = 0.0, r_net = 0.0;
    if (accept_rule == NRMG_ACCEPT_UPDATE && (s = norm_of(ctx, K, nullptr, &r_plain)) != NRMG_OK) return s;
    if ((s = copy_state(ctx, w.bP, w.bF, w.btp, Lf.P, Lf.F, Lf.tp)) != NRMG_OK) return s;  // the plain update
    CK(launch_field_correct(ctx->K, Lf, y, w.s, U, grid_for(ctx, 3, Lf.ncell), st));
    ctx->launches += 1;
    bool physical = true;
    if (accept_rule == NRMG_ACCEPT_UPDATE) {
      s = norm_of(ctx, K, nullptr, &r_net);  // a non-physical candidate reports here (status cleared)
      if (s != NRMG_OK && s != NRMG_ERR_NONPHYSICAL) return s;
      physical = s == NRMG_OK;
      accepted = physical && isfinite(r_net) && r_net < r_plain;
    } else {
      if ((s = sync_status(ctx)) != NRMG_OK && s != NRMG_ERR_NONPHYSICAL) return s;
      physical = s == NRMG_OK;
      accepted = physical;
      if (physical && accept_rule == NRMG_ACCEPT_SMOOTHED) {
        // smooth the candidate, keep it aside, smooth the plain update, compare
        s = smooth_level(ctx, K, o.s2);
        if (s == NRMG_OK) s = norm_of(ctx, K, nullptr, &r_net);
        if (s != NRMG_OK && s != NRMG_ERR_NONPHYSICAL && s != NRMG_ERR_TIMEOUT) return s;
        accepted = s == NRMG_OK && isfinite(r_net);
        if (accepted && (s = copy_state(ctx, w.cP, w.cF, w.ctp, Lf.P, Lf.F, Lf.tp)) != NRMG_OK) return s;
        if ((s = copy_state(ctx, Lf.P, Lf.F, Lf.tp, w.bP, w.bF, w.btp)) != NRMG_OK) return s;
        if ((s = smooth_level(ctx, K, o.s2)) != NRMG_OK) return s;
        if ((s = norm_of(ctx, K, nullptr, &r_plain)) != NRMG_OK) return s;
        accepted = accepted && r_net < r_plain;
        if (accepted && (s = copy_state(ctx, Lf.P, Lf.F, Lf.tp, w.cP, w.cF, w.ctp)) != NRMG_OK) return s;
        smoothed = true;
      }
    }
    if (!accepted && !smoothed && (s = copy_state(ctx, Lf.P, Lf.F, Lf.tp, w.bP, w.bF, w.btp)) != NRMG_OK) return s;
  }
  if (!smoothed && (s = smooth_level(ctx, K, o.s2)) != NRMG_OK) return s;
  if ((s = mass_correct(ctx)) != NRMG_OK) return s;
  double r = 0.0;
  if ((s = norm_of(ctx, K, nullptr, &r)) != NRMG_OK) return s;
  if (rel_res_out) *rel_res_out = ctx->res0 > 0.0 ? r / ctx->res0 : 0.0;
  if (accepted_out) *accepted_out = accepted;
  if (scale_out) {
    CK(cudaMemcpyAsync(ctx->hpin, w.s, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *scale_out = ctx->hpin[0];
  }
  return NRMG_OK;
}

nrmg_status nrmg_learned_correct(nrmg_ctx *ctx, const float *dev_y, double scale, double U) {
  if (!ctx || !dev_y || !(scale > 0.0) || !(U > 0.0) || !isfinite(scale * U)) return NRMG_ERR_ARG;
  LevelDev &Lf = ctx->lev[ctx->levels - 1];
  ctx->hpin[0] = scale;
  CK(cudaMemcpyAsync(ctx->dscal + 16, ctx->hpin, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(launch_field_correct(ctx->K, Lf, dev_y, ctx->dscal + 16, U, grid_for(ctx, 3, Lf.ncell), ctx->stream));
  ctx->launches += 1;
  return sync_status(ctx);
}

nrmg_status nrmg_solve(nrmg_ctx *ctx, double tol, int max_cycles, int *cycles_out, double *rel_res_out) {
  if (!ctx || !(tol >= 0.0) || max_cycles < 0) return NRMG_ERR_ARG;
  const int K = ctx->levels - 1;
  ctx->lev[K].has_r = 0;
  double rr = 0.0;
  nrmg_status s;
  // precision 1: every norm of the solve also leaves the defect of its state, which the next
  // cycle's first finest-level smoothing takes instead of evaluating it again
  const bool mixed = ctx->opts.precision == 1;
  if (ctx->ref_fixed) {
    if ((s = norm_of(ctx, K, nullptr, &rr, mixed)) != NRMG_OK) return s;
    rr = ctx->res0 > 0.0 ? rr / ctx->res0 : 0.0;
  } else {
    if ((s = norm_of(ctx, K, nullptr, &ctx->res0, mixed)) != NRMG_OK) return s;
    ctx->have_res0 = 1;
    rr = ctx->res0 > 0.0 ? 1.0 : 0.0;
  }
  // precision 1: stall test on the running minimum of the relative residual
  constexpr int kStallWindow = 8;
  constexpr double kStallDrop = 0.8;
  double best[kStallWindow + 1];
  ctx->mixed_off = 0;
  ctx->mixed_stalled = 0;
  int it = 0;
  while (rr > tol && it < max_cycles) {
    if ((s = fas_cycle(ctx, &rr, mixed, mixed)) != NRMG_OK) break;
    ++it;
    if (ctx->opts.precision == 1 && !ctx->mixed_off) {
      const double b = it == 1 ? rr : std::min(rr, best[(it - 1) % (kStallWindow + 1)]);
      if (it > kStallWindow && b > kStallDrop * best[(it - kStallWindow) % (kStallWindow + 1)]) ctx->mixed_off = 1;
      best[it % (kStallWindow + 1)] = b;
    }
  }
  ctx->mixed_stalled = ctx->mixed_off;
  ctx->mixed_off = 0;
  if (cycles_out) *cycles_out = it;
  if (rel_res_out) *rel_res_out = rr;
  if (s == NRMG_OK && rr > tol) s = NRMG_ERR_NOT_CONVERGED;
  return s;
}

int nrmg_mixed_fallback(const nrmg_ctx *ctx) { return ctx ? ctx->mixed_stalled : 0; }

nrmg_status nrmg_fields(nrmg_ctx *ctx, double *dev_out) {
  if (!ctx || !dev_out) return NRMG_ERR_ARG;
  CK(launch_fields(ctx->K, ctx->lev[ctx->levels - 1], dev_out, ctx->stream));
  ctx->launches += 1;
  return NRMG_OK;
}

nrmg_status nrmg_two_grid_setup(nrmg_ctx *ctx, int lf) {
  if (!ctx || lf < 1 || lf >= ctx->levels) return NRMG_ERR_ARG;
  return two_grid_setup(ctx, lf);
}

nrmg_status nrmg_two_grid_update(nrmg_ctx *ctx, int lf) {
  if (!ctx || lf < 1 || lf >= ctx->levels) return NRMG_ERR_ARG;
  return two_grid_update(ctx, lf);
}

nrmg_status nrmg_mass_correct(nrmg_ctx *ctx) {
  if (!ctx) return NRMG_ERR_ARG;
  return mass_correct(ctx);
}

nrmg_status nrmg_debug_stalled_sweep(nrmg_ctx *ctx, int level) {
  if (!ctx || level < 0 || level >= ctx->levels) return NRMG_ERR_ARG;
  LevelDev &L = ctx->lev[level];
  // every update counter starts far below any version an update waits for: nothing ever
  // satisfies the first wait, which runs out after its time limit
  CK(cudaMemsetAsync(L.ver, 0x80, sizeof(int) * L.ncell, ctx->stream));
  CK(cudaMemsetAsync(ctx->K.queue, 0, sizeof(int), ctx->stream));
  int g = grid_for(ctx, 0, 4LL * L.ncell);
  CK(launch_fs(ctx->K, L, 1, nullptr, g, ctx->stream));
  ctx->launches += 1;
  return sync_status(ctx);
}

nrmg_status nrmg_sync(nrmg_ctx *ctx) {
  if (!ctx) return NRMG_ERR_ARG;
  return sync_status(ctx);
}

long long nrmg_launch_count(const nrmg_ctx *ctx) { return ctx ? ctx->launches : 0; }

nrmg_status nrmg_set_profiling(nrmg_ctx *ctx, int on) {
  if (!ctx) return NRMG_ERR_ARG;
  if (on && ctx->ev.empty()) {
    const size_t n = 2 * 65536;
    ctx->ev.resize(n);
    for (size_t k = 0; k < n; ++k) CK(cudaEventCreate(&ctx->ev[k]));
    ctx->ev_upd.assign(n / 2, 0);
    ctx->ev_hasr.assign(n / 2, 0);
    ctx->ev_level.assign(n / 2, 0);
    ctx->ev_prec.assign(n / 2, 0);
    const size_t nr = 2 * 16384;
    ctx->rev.resize(nr);
    for (size_t k = 0; k < nr; ++k) CK(cudaEventCreate(&ctx->rev[k]));
    ctx->rev_cells.assign(nr / 2, 0);
    ctx->rev_hasr.assign(nr / 2, 0);
  }
  ctx->profiling = on ? 1 : 0;
  ctx->ev_used = 0;
  ctx->rev_used = 0;
  return NRMG_OK;
}

nrmg_status nrmg_residual_profile(nrmg_ctx *ctx, double *ms, long long *launches, long long *cells_no_r,
                                  long long *cells_r) {
  if (!ctx) return NRMG_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  double tot = 0.0;
  long long c0 = 0, c1 = 0;
  for (size_t k = 0; k + 1 < ctx->rev_used; k += 2) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, ctx->rev[k], ctx->rev[k + 1]));
    tot += t;
    if (ctx->rev_hasr[k / 2])
      c1 += ctx->rev_cells[k / 2];
    else
      c0 += ctx->rev_cells[k / 2];
  }
  if (ms) *ms = tot;
  if (launches) *launches = (long long)(ctx->rev_used / 2);
  if (cells_no_r) *cells_no_r = c0;
  if (cells_r) *cells_r = c1;
  ctx->rev_used = 0;
  return NRMG_OK;
}

nrmg_status nrmg_fs_profile_levels(nrmg_ctx *ctx, double *ms_per_level, long long *updates_per_level) {
  if (!ctx || !ms_per_level || !updates_per_level) return NRMG_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  for (int l = 0; l < ctx->levels; ++l) {
    ms_per_level[l] = 0.0;
    updates_per_level[l] = 0;
  }
  for (size_t k = 0; k + 1 < ctx->ev_used; k += 2) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, ctx->ev[k], ctx->ev[k + 1]));
    ms_per_level[ctx->ev_level[k / 2]] += t;
    updates_per_level[ctx->ev_level[k / 2]] += ctx->ev_upd[k / 2];
  }
  return NRMG_OK;
}

nrmg_status nrmg_fs_profile(nrmg_ctx *ctx, double *ms, long long *launches, long long *updates_no_r,
                            long long *updates_r) {
  if (!ctx) return NRMG_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  double tot = 0.0;
  long long u0 = 0, u1 = 0;
  for (size_t k = 0; k + 1 < ctx->ev_used; k += 2) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, ctx->ev[k], ctx->ev[k + 1]));
    tot += t;
    if (ctx->ev_hasr[k / 2])
      u1 += ctx->ev_upd[k / 2];
    else
      u0 += ctx->ev_upd[k / 2];
  }
  if (ms) *ms = tot;
  if (launches) *launches = (long long)(ctx->ev_used / 2);
  if (updates_no_r) *updates_no_r = u0;
  if (updates_r) *updates_r = u1;
  ctx->ev_used = 0;
  return NRMG_OK;
}

const char *nrmg_status_str(nrmg_status s) {
  switch (s) {
    case NRMG_OK: return "NRMG_OK";
    case NRMG_ERR_ARG: return "NRMG_ERR_ARG";
    case NRMG_ERR_CUDA: return "NRMG_ERR_CUDA";
    case NRMG_ERR_OOM: return "NRMG_ERR_OOM";
    case NRMG_ERR_NONPHYSICAL: return "NRMG_ERR_NONPHYSICAL";
    case NRMG_ERR_NOT_CONVERGED: return "NRMG_ERR_NOT_CONVERGED";
    case NRMG_ERR_TIMEOUT: return "NRMG_ERR_TIMEOUT";
  }
  return "NRMG_UNKNOWN";
}

const char *nrmg_last_error(const nrmg_ctx *ctx) { return ctx ? ctx->err : ""; }

}  // extern "C"

// ------------------------------------------------------------------ batches of problems
// A batch runs the V-cycles of several problems in lockstep, aligned by depth below each
// problem's finest level.  Every FS stage (the pre-smoothing at one depth, the coarsest
// solves reached at that depth, the post-smoothing at one depth) of all problems is one
// persistent launch whose queue merges the problems' dependency-graph schedules by start time.
struct nrmg_batch {
  std::vector<nrmg_ctx *> ctx;
  cudaStream_t stream;
  struct Stage {
    int ndesc;
    BatchDesc *desc;        // device
    int2 *items;            // device
    long long nitems;
    std::vector<std::pair<int, int>> ver;  // (problem, level) whose counters are reset
  };
  std::vector<Stage> down, up;  // down[d]: depth d pre-smoothing / coarsest; up[d]: depth d post
  int *ctl;                     // device: [0] item counter, [1] abort word
  int kmax;                     // the context of the largest M (shared-memory layout, occupancy)
  int grid;
  int depth;
  long long launches;
  // the batched cycle captured as a CUDA graph (after one eager cycle; legacy default stream:
  // never captured)
  int cycles_run;
  int graph_state;  // 0 not tried, 1 replaying, 2 capture unavailable
  cudaGraphExec_t gexec;
  int graph_grid;
  long long graph_launches;
  char err[256];
};

namespace {

bool batch_compatible(nrmg_ctx *const *c, int n) {
  if (!c || n < 1) return false;
  for (int b = 0; b < n; ++b) {
    if (!c[b]) return false;
    const nrmg_opts &o = c[b]->opts, &o0 = c[0]->opts;
    if (o.order != o0.order || o.slope != o0.slope || o.s1 != o0.s1 || o.s2 != o0.s2 ||
        o.s3 != o0.s3 || o.gamma != 1 || o.precision != 0 || c[b]->coll.model != c[0]->coll.model)
      return false;
  }
  return true;
}

// the FS stages of a batched V-cycle; ws == nullptr only sizes them
size_t batch_stages(nrmg_ctx *const *c, int n, char *ws, nrmg_batch *B) {
  int D = 0;
  for (int b = 0; b < n; ++b) D = std::max(D, c[b]->levels - 1);
  size_t off = 256;  // control words first
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~size_t(255);
    size_t o = off;
    off += bytes;
    return o;
  };
  for (int pass = 0; pass < 2; ++pass) {
    for (int d = (pass == 0 ? 0 : D - 1); pass == 0 ? d <= D : d >= 0; d += (pass == 0 ? 1 : -1)) {
      // entries of this stage: (problem, level, steps)
      std::vector<int> eb, el, es;
      for (int b = 0; b < n; ++b) {
        int l = c[b]->levels - 1 - d;
        if (pass == 0 && l >= 0) {
          eb.push_back(b);
          el.push_back(l);
          es.push_back(l == 0 ? c[b]->opts.s3 : c[b]->opts.s1);
        } else if (pass == 1 && l >= 1) {
          eb.push_back(b);
          el.push_back(l);
          es.push_back(c[b]->opts.s2);
        }
      }
      long long nit = 0;
      for (size_t e = 0; e < eb.size(); ++e) nit += (long long)es[e] * 4 * c[eb[e]]->lev[el[e]].ncell;
      size_t od = take(sizeof(BatchDesc) * eb.size()), oi = take(sizeof(int2) * (size_t)nit);
      if (!ws) continue;
      nrmg_batch::Stage S;
      S.ndesc = (int)eb.size();
      S.desc = (BatchDesc *)(ws + od);
      S.items = (int2 *)(ws + oi);
      S.nitems = nit;
      std::vector<BatchDesc> hd(eb.size());
      std::vector<std::pair<long long, int2>> all;
      all.reserve(nit);
      for (size_t e = 0; e < eb.size(); ++e) {
        nrmg_ctx *x = c[eb[e]];
        hd[e].K = x->K;
        hd[e].K.abort_flag = B->ctl + 1;
        hd[e].L = x->lev[el[e]];
        hd[e].L.has_r = el[e] < x->levels - 1 ? 1 : 0;
        S.ver.push_back({eb[e], el[e]});
        std::vector<std::pair<int, int>> keys;
        asap_schedule_keys(hd[e].L.nx, hd[e].L.ny, x->K.reach, es[e], keys);
        for (auto &kv : keys) all.push_back({(long long)kv.first, make_int2((int)e, kv.second)});
      }
      std::stable_sort(all.begin(), all.end(),
                       [](const std::pair<long long, int2> &a, const std::pair<long long, int2> &b) {
                         return a.first < b.first;
                       });
      std::vector<int2> hi(all.size());
      for (size_t q = 0; q < all.size(); ++q) hi[q] = all[q].second;
      cudaMemcpyAsync(S.desc, hd.data(), sizeof(BatchDesc) * hd.size(), cudaMemcpyHostToDevice, B->stream);
      cudaMemcpyAsync(S.items, hi.data(), sizeof(int2) * hi.size(), cudaMemcpyHostToDevice, B->stream);
      cudaStreamSynchronize(B->stream);
      (pass == 0 ? B->down : B->up).push_back(S);
    }
  }
  return off + 256;
}

nrmg_status batch_fs(nrmg_batch *B, nrmg_batch::Stage &S) {
  nrmg_ctx *ctx = B->ctx[0];  // for CK's error message
  if (S.nitems == 0) return NRMG_OK;
  for (auto &bl : S.ver) {
    LevelDev &L = B->ctx[bl.first]->lev[bl.second];
    CK(cudaMemsetAsync(L.ver, 0, sizeof(int) * L.ncell, B->stream));
  }
  CK(cudaMemsetAsync(B->ctl, 0, sizeof(int), B->stream));
  long long g = std::min<long long>(B->grid, S.nitems);
  Consts K0 = B->ctx[B->kmax]->K;  // the largest M: shared-memory size and first tables
  K0.abort_flag = B->ctl + 1;
  CK(launch_fs_batch(S.desc, S.items, S.nitems, B->ctl, K0, (int)g, B->stream));
  B->launches += 1;
  return NRMG_OK;
}

// one batched V-cycle with mass correction; the norms are left in each context's dscal[0]
nrmg_status batch_cycle_async(nrmg_batch *B) {
  const int n = (int)B->ctx.size();
  nrmg_status s;
  // work of the contexts goes to the batch stream
  std::vector<cudaStream_t> saved(n);
  for (int b = 0; b < n; ++b) {
    saved[b] = B->ctx[b]->stream;
    B->ctx[b]->stream = B->stream;
    B->ctx[b]->lev[B->ctx[b]->levels - 1].has_r = 0;
  }
  auto restore = [&]() {
    for (int b = 0; b < n; ++b) B->ctx[b]->stream = saved[b];
  };
  for (int d = 0; d <= B->depth; ++d) {
    if ((s = batch_fs(B, B->down[d])) != NRMG_OK) return restore(), s;
    for (int b = 0; b < n; ++b) {
      int l = B->ctx[b]->levels - 1 - d;
      if (l >= 1 && (s = two_grid_setup(B->ctx[b], l)) != NRMG_OK) return restore(), s;
    }
  }
  for (int d = B->depth - 1, u = 0; d >= 0; --d, ++u) {
    for (int b = 0; b < n; ++b) {
      int l = B->ctx[b]->levels - 1 - d;
      if (l >= 1 && (s = two_grid_update(B->ctx[b], l)) != NRMG_OK) return restore(), s;
    }
    if ((s = batch_fs(B, B->up[u])) != NRMG_OK) return restore(), s;
  }
  for (int b = 0; b < n; ++b) {
    nrmg_ctx *ctx = B->ctx[b];
    if ((s = mass_correct(ctx)) != NRMG_OK) return restore(), s;
    int g = 0;
    if ((s = residual(ctx, ctx->levels - 1, kResOut, nullptr, ctx->N, &g)) != NRMG_OK) return restore(), s;
    cudaError_t e = launch_reduce_norm(ctx->partials, g, 1.0 / (ctx->grid.lx * ctx->grid.ly), ctx->dscal, B->stream);
    if (e != cudaSuccess) return restore(), NRMG_ERR_CUDA;
    ctx->launches += 1;
  }
  restore();
  return NRMG_OK;
}

nrmg_status batch_norms(nrmg_batch *B, std::vector<double> &out) {
  const int n = (int)B->ctx.size();
  out.assign(n, 0.0);
  std::vector<int> st(n, 0);
  for (int b = 0; b < n; ++b) {
    if (cudaMemcpyAsync(&out[b], B->ctx[b]->dscal, sizeof(double), cudaMemcpyDeviceToHost, B->stream) != cudaSuccess)
      return NRMG_ERR_CUDA;
    if (cudaMemcpyAsync(&st[b], B->ctx[b]->dstatus, sizeof(int), cudaMemcpyDeviceToHost, B->stream) != cudaSuccess)
      return NRMG_ERR_CUDA;
  }
  if (cudaStreamSynchronize(B->stream) != cudaSuccess) return NRMG_ERR_CUDA;
  for (int b = 0; b < n; ++b)
    if (st[b] != 0) {
      cudaMemsetAsync(B->ctx[b]->dstatus, 0, 2 * sizeof(int), B->stream);
      cudaMemsetAsync(B->ctl, 0, 2 * sizeof(int), B->stream);
      cudaStreamSynchronize(B->stream);
      snprintf(B->err, sizeof(B->err), "problem %d reported status %d", b, st[b]);
      return (nrmg_status)st[b];
    }
  return NRMG_OK;
}

}  // namespace

extern "C" {

size_t nrmg_batch_workspace_bytes(nrmg_ctx *const *ctxs, int n) {
  if (!batch_compatible(ctxs, n)) return 0;
  return batch_stages(ctxs, n, nullptr, nullptr);
}

nrmg_status nrmg_batch_create(nrmg_ctx *const *ctxs, int n, void *dev_workspace, size_t ws_bytes,
                              nrmg_batch **out) {
  if (!out) return NRMG_ERR_ARG;
  *out = nullptr;
  if (!batch_compatible(ctxs, n) || !dev_workspace || ((uintptr_t)dev_workspace & 255)) return NRMG_ERR_ARG;
  size_t need = nrmg_batch_workspace_bytes(ctxs, n);
  if (ws_bytes < need) return NRMG_ERR_OOM;
  nrmg_batch *B = new nrmg_batch();
  B->ctx.assign(ctxs, ctxs + n);
  B->stream = ctxs[0]->stream;
  B->ctl = (int *)dev_workspace;
  B->launches = 0;
  B->cycles_run = 0;
  B->graph_state = 0;
  B->gexec = nullptr;
  B->graph_grid = 0;
  B->graph_launches = 0;
  B->err[0] = 0;
  int D = 0;
  for (int b = 0; b < n; ++b) D = std::max(D, ctxs[b]->levels - 1);
  B->depth = D;
  B->kmax = 0;
  for (int b = 1; b < n; ++b)
    if (ctxs[b]->M > ctxs[B->kmax]->M) B->kmax = b;
  B->grid = ctxs[0]->nsm * std::max(1, ctxs[B->kmax]->occ[0]);
  if (cudaMemsetAsync(B->ctl, 0, 256, B->stream) != cudaSuccess) {
    delete B;
    return NRMG_ERR_CUDA;
  }
  batch_stages(ctxs, n, (char *)dev_workspace, B);
  if (cudaStreamSynchronize(B->stream) != cudaSuccess) {
    delete B;
    return NRMG_ERR_CUDA;
  }
  *out = B;
  return NRMG_OK;
}

nrmg_status nrmg_batch_destroy(nrmg_batch *B) {
  if (!B) return NRMG_ERR_ARG;
  cudaStreamSynchronize(B->stream);
  if (B->gexec) cudaGraphExecDestroy(B->gexec);
  delete B;
  return NRMG_OK;
}

nrmg_status nrmg_batch_fas_cycle(nrmg_batch *B, double *rel_res_out) {
  if (!B) return NRMG_ERR_ARG;
  const int n = (int)B->ctx.size();
  nrmg_status s;
  std::vector<double> nr;
  // reference residuals of the problems that have none yet
  for (int b = 0; b < n; ++b) {
    nrmg_ctx *ctx = B->ctx[b];
    if (!ctx->have_res0) {
      ctx->lev[ctx->levels - 1].has_r = 0;
      if ((s = norm_of(ctx, ctx->levels - 1, nullptr, &ctx->res0)) != NRMG_OK) return s;
      ctx->have_res0 = 1;
    }
  }
  if (B->graph_state == 1 && B->graph_grid != B->grid) {  // the grid changed: capture again
    cudaGraphExecDestroy(B->gexec);
    B->gexec = nullptr;
    B->graph_state = 0;
  }
  if (B->graph_state == 1) {
    if (cudaGraphLaunch(B->gexec, B->stream) != cudaSuccess) return NRMG_ERR_CUDA;
    B->launches += B->graph_launches;
  } else if (B->graph_state == 0 && B->cycles_run >= 1 && B->stream != nullptr) {
    // capture this cycle; fall back to eager launches if capture is not possible
    long long before = nrmg_batch_launch_count(B);
    bool captured = false;
    if (cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      s = batch_cycle_async(B);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(B->stream, &g);
      if (s == NRMG_OK && e == cudaSuccess && g &&
          cudaGraphInstantiate(&B->gexec, g, 0) == cudaSuccess) {
        captured = true;
        B->graph_launches = nrmg_batch_launch_count(B) - before;
        B->graph_grid = B->grid;
      }
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
    if (captured) {
      B->graph_state = 1;
      if (cudaGraphLaunch(B->gexec, B->stream) != cudaSuccess) return NRMG_ERR_CUDA;
    } else {
      B->graph_state = 2;
      if ((s = batch_cycle_async(B)) != NRMG_OK) return s;
    }
  } else {
    if ((s = batch_cycle_async(B)) != NRMG_OK) return s;
  }
  B->cycles_run += 1;
  if ((s = batch_norms(B, nr)) != NRMG_OK) return s;
  if (rel_res_out)
    for (int b = 0; b < n; ++b) rel_res_out[b] = B->ctx[b]->res0 > 0.0 ? nr[b] / B->ctx[b]->res0 : 0.0;
  return NRMG_OK;
}

nrmg_status nrmg_batch_solve(nrmg_batch *B, double tol, int max_cycles, int *cycles_out, double *rel_res_out) {
  if (!B || !(tol >= 0.0) || max_cycles < 0) return NRMG_ERR_ARG;
  const int n = (int)B->ctx.size();
  std::vector<double> rel(n, 1.0);
  std::vector<int> cyc(n, 0);
  nrmg_status s = NRMG_OK;
  for (int b = 0; b < n; ++b) {
    nrmg_ctx *ctx = B->ctx[b];
    ctx->lev[ctx->levels - 1].has_r = 0;
    if (ctx->ref_fixed) {
      double r = 0.0;
      if ((s = norm_of(ctx, ctx->levels - 1, nullptr, &r)) != NRMG_OK) return s;
      rel[b] = ctx->res0 > 0.0 ? r / ctx->res0 : 0.0;
      continue;
    }
    if ((s = norm_of(ctx, ctx->levels - 1, nullptr, &ctx->res0)) != NRMG_OK) return s;
    ctx->have_res0 = 1;
    rel[b] = ctx->res0 > 0.0 ? 1.0 : 0.0;
  }
  auto done = [&]() {
    for (int b = 0; b < n; ++b)
      if (rel[b] > tol) return false;
    return true;
  };
  int it = 0;
  while (!done() && it < max_cycles) {
    std::vector<double> r(n);
    if ((s = nrmg_batch_fas_cycle(B, r.data())) != NRMG_OK) break;
    ++it;
    for (int b = 0; b < n; ++b)
      if (rel[b] > tol) {
        rel[b] = r[b];
        cyc[b] = it;
      }
  }
  if (cycles_out)
    for (int b = 0; b < n; ++b) cycles_out[b] = cyc[b];
  if (rel_res_out)
    for (int b = 0; b < n; ++b) rel_res_out[b] = rel[b];
  if (s == NRMG_OK && !done()) s = NRMG_ERR_NOT_CONVERGED;
  return s;
}

int nrmg_batch_graph(const nrmg_batch *B) { return B && B->graph_state == 1 ? 1 : 0; }

nrmg_status nrmg_batch_set_grid(nrmg_batch *B, int ctas_per_sm) {
  if (!B || ctas_per_sm < 1 || ctas_per_sm > std::max(1, B->ctx[B->kmax]->occ[0])) return NRMG_ERR_ARG;
  B->grid = B->ctx[0]->nsm * ctas_per_sm;
  return NRMG_OK;
}

long long nrmg_batch_launch_count(const nrmg_batch *B) {
  if (!B) return 0;
  long long n = B->launches;
  for (nrmg_ctx *c : B->ctx) n += c->launches;
  return n;
}

}  // extern "C"

// ------------------------------------------------------------------ residual without allocation
// Scratch of nrmg_residual_noalloc: a file-scope device array, so that callers who cannot
// allocate device memory (no cudaMalloc, no caching allocator, no workspace of their own) can
// still evaluate a residual.  Every GPU that loads the library holds it until the process exits.
#define NRMG_NOALLOC_SCRATCH_BYTES (16u << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[NRMG_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of the scratch array on the current device.  In host code the array's name
// is only a host-side stand-in, so the address is looked up with the device current; it is
// looked up on every call (no allocation, no cache shared between host threads, and still
// right after the device's context was reset).
cudaError_t noalloc_scratch(void **out) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

}  // namespace

extern "C" nrmg_status nrmg_residual_noalloc(const nrmg_grid *grid, int M, double Kn, const nrmg_wall walls[4],
                                             const nrmg_collision *coll, const nrmg_opts *opts,
                                             const double *dev_params, const double *dev_coeffs, double *dev_R_out,
                                             double *norm_out, void *cuda_stream) {
  if (!grid_ok(grid) || M < 3 || M > kMaxM || !(Kn > 0.0) || !walls || !coll || !opts_ok(opts) || !dev_params ||
      !dev_coeffs)
    return NRMG_ERR_ARG;
  if (coll->model != NRMG_BGK && coll->model != NRMG_SHAKHOV && coll->model != NRMG_ESBGK) return NRMG_ERR_ARG;
  if (!(coll->beta > 0.0) || !(coll->Pr > 0.0) || !isfinite(coll->omega)) return NRMG_ERR_ARG;
  for (int w = 0; w < 4; ++w) {
    if (!(walls[w].theta > 0.0) || walls[w].chi < 0.0 || walls[w].chi > 1.0) return NRMG_ERR_ARG;
    if (walls[w].u[kWallAxis[w]] != 0.0 || walls[w].u[2] != 0.0) return NRMG_ERR_ARG;
  }
  const int N = nmom(M), NP = pad4(N), NE = nmom_even(M);
  const long long ncell = (long long)grid->nx * grid->ny;
  // layout of the scratch: tables, control words, reduction scratch, padded copy of the state
  size_t used = 0;
  auto at = [&](size_t bytes) {
    used = (used + 255) & ~size_t(255);
    size_t o = used;
    used += bytes;
    return o;
  };
  const size_t o_i32 = at(tab_i32_size(M) * sizeof(int32_t));
  const size_t o_u16 = at((13 * N + NE) * sizeof(uint16_t));
  const size_t o_f64 = at(N * sizeof(double));
  const size_t o_W = at(4 * (M + 1) * (M + 1) * sizeof(double));
  const size_t o_R = at(4 * (M + 1) * sizeof(double));
  const size_t o_In = at(4 * (M + 1) * sizeof(double));
  const size_t o_ctl = at(64 * sizeof(int));
  const size_t o_part = at(kPartials * sizeof(double));
  const size_t o_scal = at(64 * sizeof(double));
  const size_t o_P = at(ncell * 4 * sizeof(double));
  const size_t o_F = at(ncell * NP * sizeof(double));
  const size_t o_tp = at(ncell * sizeof(double));
  if (used > NRMG_NOALLOC_SCRATCH_BYTES) return NRMG_ERR_OOM;

  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  void *base = nullptr;
  if (cudaGetDevice(&dev) != cudaSuccess) return NRMG_ERR_CUDA;
  if (noalloc_scratch(&base) != cudaSuccess) return NRMG_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NRMG_ERR_CUDA;
  char *b = (char *)base;

  Consts K;
  memset(&K, 0, sizeof(K));
  K.M = M;
  K.N = N;
  K.NP = NP;
  K.NE = NE;
  K.iq_off = 3 * NE + N;
  K.ln_off = K.iq_off + 18;
  for (int d = 0; d < 3; ++d) K.nl[d] = nlines(M, d);
  K.reach = (opts->order == 2 && opts->slope != 0) ? 2 : 1;
  K.slope = opts->order == 2 ? opts->slope : 0;
  K.model = coll->model;
  K.Kn = Kn;
  K.Pr = coll->Pr;
  K.omega = coll->omega;
  K.beta = coll->beta;
  K.cfl = opts->cfl;
  K.dtnu = opts->dtnu;
  K.nu0 = coll->beta * sqrt(M_PI / 2.0) / Kn;
  K.C = hermite_largest_root(M + 1);
  K.lx = grid->lx;
  K.ly = grid->ly;
  for (int w = 0; w < 4; ++w) {
    for (int d = 0; d < 3; ++d) K.wall_u[w][d] = walls[w].u[d];
    K.wall_theta[w] = walls[w].theta;
  }
  Tables T;
  build_tables(M, T);
  memcpy(K.idx_axis, T.idx_axis, sizeof(T.idx_axis));
  memcpy(K.idx_e, T.idx_e, sizeof(T.idx_e));
  memcpy(K.idx_2e, T.idx_2e, sizeof(T.idx_2e));
  std::vector<double> W, R, In;
  wall_tables(M, walls, W, R, In);
  K.tab_i32 = (const int *)(b + o_i32);
  K.tab_u16 = (const uint16_t *)(b + o_u16);
  K.tab_f64 = (const double *)(b + o_f64);
  K.wallW = (const double *)(b + o_W);
  K.wallRho = (const double *)(b + o_R);
  K.wallIn = (const double *)(b + o_In);
  K.status = (int *)(b + o_ctl);
  K.abort_flag = K.status + 1;
  K.queue = K.status + 2;
  double *partials = (double *)(b + o_part), *scal = (double *)(b + o_scal);

  LevelDev L;
  memset(&L, 0, sizeof(L));
  L.nx = grid->nx;
  L.ny = grid->ny;
  L.ncell = (int)ncell;
  L.dx = grid->lx / grid->nx;
  L.dy = grid->ly / grid->ny;
  L.idx = 1.0 / L.dx;
  L.idy = 1.0 / L.dy;
  L.P = (double *)(b + o_P);
  L.F = (double *)(b + o_F);
  L.tp = (double *)(b + o_tp);
  L.has_r = 0;
  L.uniform = 1;

#define NA(expr)                                  \
  do {                                            \
    if ((expr) != cudaSuccess) return NRMG_ERR_CUDA; \
  } while (0)
  NA(cudaMemcpyAsync((void *)K.tab_i32, T.i32.data(), T.i32.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  NA(cudaMemcpyAsync((void *)K.tab_u16, T.u16.data(), T.u16.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, st));
  NA(cudaMemcpyAsync((void *)K.tab_f64, T.fact.data(), T.fact.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  NA(cudaMemcpyAsync((void *)K.wallW, W.data(), W.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  NA(cudaMemcpyAsync((void *)K.wallRho, R.data(), R.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  NA(cudaMemcpyAsync((void *)K.wallIn, In.data(), In.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  // the status words must start at zero; everything else is overwritten before it is read
  NA(cudaMemsetAsync(K.status, 0, 64 * sizeof(int), st));
  NA(cudaMemcpyAsync(L.P, dev_params, sizeof(double) * 4 * ncell, cudaMemcpyDeviceToDevice, st));
  NA(launch_pack(dev_coeffs, N, L.F, NP, L.ncell, N, st));
  NA(launch_check_state(K, L.P, L.F, NP, L.ncell, 0, st));
  NA(launch_tpow(K, L, st));
  int occ = occupancy_cell(M, NP, 1);
  long long g = (long long)nsm * (occ < 1 ? 1 : occ);
  if (g > ncell) g = ncell;
  if (g > kPartials) g = kPartials;
  NA(launch_residual(K, L, kResOut, dev_R_out, N, partials, (int)g, st));
  NA(launch_reduce_norm(partials, (int)g, 1.0 / (grid->lx * grid->ly), scal, st));
  double hnorm = 0.0;
  int hstatus = 0;
  NA(cudaMemcpyAsync(&hnorm, scal, sizeof(double), cudaMemcpyDeviceToHost, st));
  NA(cudaMemcpyAsync(&hstatus, K.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  NA(cudaStreamSynchronize(st));
#undef NA
  if (hstatus != 0) return (nrmg_status)hstatus;
  if (norm_out) *norm_out = hnorm;
  return NRMG_OK;
}
