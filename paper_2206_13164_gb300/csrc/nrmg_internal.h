// Internal declarations shared by the host (C ABI) and device translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct nrmg_net;

namespace nrmg {

constexpr int kMaxM = 16;
constexpr int kMaxN = 969;   // C(19,3)
constexpr int kMaxLev = 16;
constexpr int kNV = 9;       // transform vectors per cell update: 4 faces x 2 sides + r
constexpr int kThreads = 256;

// Device status codes (same values as nrmg_status).
constexpr int kStOk = 0, kStNonPhysical = 4, kStTimeout = 6;

// Kernel modes of the Jacobi-style residual kernel.
enum ResMode { kResOut = 0, kResDefect = 1, kResCoarseRhs = 2, kResDefectNorm = 3 };

struct LevelDev {
  int nx, ny, ncell;
  double dx, dy;
  double idx, idy;  // 1/dx, 1/dy
  double *P, *F;    // state: [ncell][4], [ncell][NP]
  double *rP, *rF;  // right-hand side r and its expansion bases
  double *bP, *bF;  // restricted state saved for the coarse-grid update
  double *D;        // defect r - R(f)
  double *tp;       // theta^(1-omega) of each cell, written with the cell's state
  int *ver;         // per-cell update counters of the sweep scheduler
  int *order;       // [4][ncell]: cells of sweep Dk in anti-diagonal order
  int has_r;
  // FP32 correction sweeps (precision 1): correction e, each coefficient in one 64-bit word
  // with the version of the update that wrote it (low half the float, high half the version),
  // FP64 defect rounded to FP32, and the frozen per-cell coefficients (u1, u2, u3, theta, dt,
  // nu, 0, 0)
  unsigned long long *et;
  float *d32, *aux32;
  float *s32;  // FP32 copy of the state's coefficients: the frozen limiter weights of the correction
  // Non-uniform grid (nrmg_set_spacing; uniform = 1 leaves these NULL and uses dx, dy): widths
  // hx[nx], hy[ny] and their inverses, and per column (row) the factors of the second-order
  // reconstruction: rm = h / hm, rp = h / hp (h the cell's width, hm, hp the distances to the
  // neighbouring centres) and ch = h / (2 (hm + hp))
  int uniform;
  const double *hx, *hy, *ihx, *ihy;
  const double *rmx, *rpx, *chx, *rmy, *rpy, *chy;
};

// Everything a kernel needs besides the level: scheme constants and
// pointers to the index tables built by the host.
struct Consts {
  int M, N, NP;
  int NE;      // number of multi-indices with even alpha_3 (the only nonzero ones of a planar state)
  int iq_off;  // offset in tab_i32 of the heat-flux and stress indices
  int ln_off;  // offset in tab_i32 of the index lines of directions 0, 1, 2 (nl[d] entries each)
  int nl[3];
  int reach;   // stencil reach: 1 (first order) or 2 (second order)
  int slope;   // 0 none, 1 central, 2 van Albada
  int model;
  double Kn, Pr, omega, beta, cfl, C;  // C = largest root of He_{M+1}
  double dtnu;                         // > 0: time step capped at dtnu / nu
  double nu0;                          // beta sqrt(pi/2) / Kn: nu = nu0 rho theta^(1-omega)
  double lx, ly;
  double wall_u[4][3], wall_theta[4];
  // tables (global memory, copied to shared memory by each CTA)
  const int *tab_i32;   // tslot[3][NE], tshak[N] (Shakhov target or -1), iq[3][4], is[6], lines
                        // (start | length << 11, longest first, per direction)
  const uint16_t *tab_u16;  // tmem[3][N], tprev[3][N], tnext[3][N] (0xFFFF = none), tal[3][N], tdeg[N], eidx[NE]
  const double *tab_f64;    // fact[N] (alpha!)
  const double *wallW;      // [4][(M+1)^2]: W^s_{k,m}
  const double *wallRho;    // [4][M+1]
  const double *wallIn;     // [4][M+1]
  const float *wallWf, *wallRf, *wallInf;  // FP32 copies of the three wall tables
  int idx_axis[2][kMaxM + 1];  // index of m e_x, m e_y
  int idx_e[3], idx_2e[3];
  int *status;
  int *abort_flag;
  int *queue;
};

// Number of multi-indices |alpha| <= M with even alpha_3.
__host__ __device__ inline int nmom_even(int M) {
  int n = 0;
  for (int a3 = 0; a3 <= M; a3 += 2) n += (M - a3 + 1) * (M - a3 + 2) / 2;
  return n;
}

// Index lines of the line-wise FP32 transform along direction d: along x and y the lines with
// even alpha_3, along alpha_3 every line (its even entries are the outputs).
__host__ __device__ inline int nlines(int M, int d) {
  if (d == 2) return (M + 1) * (M + 2) / 2;
  int n = 0;
  for (int a3 = 0; a3 <= M; a3 += 2) n += M - a3 + 1;
  return n;
}
__host__ __device__ inline int nlines_total(int M) { return nlines(M, 0) + nlines(M, 1) + nlines(M, 2); }

// One problem of a batched FS launch: its scheme constants and the level being swept.
struct BatchDesc {
  Consts K;
  LevelDev L;
};

// Size in bytes of the dynamic shared memory of the cell kernels.
size_t cell_smem_bytes(int M, int NP);

// Launchers (device translation unit).  Each returns cudaGetLastError().
// FS^steps on level L.  queue (may be NULL): the order in which the persistent CTAs take the
// steps*4*ncell items, each item (s*4 + k)*ncell + c; NULL = sweep by sweep in anti-diagonal order.
cudaError_t launch_fs(const Consts &K, const LevelDev &L, int steps, const int *queue, int grid, cudaStream_t st);
// The same sweeps with each cell update split over a cluster of two CTAs on two SMs (x faces on
// one, y faces, collision and projection on the other); nclusters persistent clusters, per_sm
// (1 or 2) CTAs per SM.
cudaError_t launch_fs_cluster(const Consts &K, const LevelDev &L, int steps, const int *queue, int nclusters,
                              int per_sm, cudaStream_t st);
// Clusters of the two-CTA sweep that fit on the device at once with per_sm CTAs per SM (0:
// cluster launch unavailable).
int cluster_capacity(const Consts &K, int per_sm);
// FS sweeps of several problems in one persistent launch (items: problem, level-queue item).
cudaError_t launch_fs_batch(const BatchDesc *desc, const int2 *items, long long total, int *counter,
                            const Consts &K0, int grid, cudaStream_t st);
cudaError_t launch_residual(const Consts &K, const LevelDev &L, int mode, double *out, int out_stride,
                            double *partials, int grid, cudaStream_t st);
cudaError_t launch_restrict(const Consts &K, const LevelDev &Lf, const LevelDev &Lc, int grid, cudaStream_t st);
cudaError_t launch_prolong(const Consts &K, const LevelDev &Lf, const LevelDev &Lc, int grid, cudaStream_t st);
// one forward Euler step (eq. euler-scheme) of a level whose L.D holds R - r of the state;
// dt_dev receives the global step
cudaError_t launch_euler(const Consts &K, const LevelDev &L, double *dt_dev, int grid, cudaStream_t st);
cudaError_t launch_reduce_norm(const double *partials, int n, double scale, double *out, cudaStream_t st);
// Total mass of level L into scal[0]; with apply, also scale every coefficient by m0 / mass
// (scal[1]).
cudaError_t launch_mass(const Consts &K, const LevelDev &L, double *partials, int grid, double *scal, double m0,
                        bool apply, cudaStream_t st);
cudaError_t launch_fields(const Consts &K, const LevelDev &L, double *out, cudaStream_t st);
// theta^(1-omega) of every cell of L (after its state was written from outside the sweeps)
cudaError_t launch_tpow(const Consts &K, const LevelDev &L, cudaStream_t st);
cudaError_t launch_pack(const double *src, int src_stride, double *dst, int dst_stride, int rows, int cols,
                        cudaStream_t st);
// Admissibility of a state (rhs = 0) or of a right-hand side (rhs = 1) handed in through the C
// ABI; records NRMG_ERR_ARG for a non-planar input, NRMG_ERR_NONPHYSICAL otherwise.
cudaError_t launch_check_state(const Consts &K, const double *P, const double *F, int stride, int ncell, int rhs,
                               cudaStream_t st);
int occupancy_cell(int M, int NP, int which);  // CTAs per SM of kernel `which` (0 fs, 1 res, 2 restrict, 3 prolong)

// FP32 correction sweeps of the mixed-precision smoother (nrmg_mixed.cu).
cudaError_t launch_mixed_prep(const Consts &K, const LevelDev &L, cudaStream_t st);
cudaError_t launch_fs_corr(const Consts &K, const LevelDev &L, int steps, const int *queue, int grid, cudaStream_t st);
cudaError_t launch_mixed_update(const Consts &K, const LevelDev &L, int grid, cudaStream_t st);
int occupancy_corr(int M, int NP);

// 13-moment Grad state of given fields (nrmg_net.cu): P [ncell][4], F [ncell][NP] in graded order.
cudaError_t launch_grad13(const double *fields, int ncell, int M, int NP, double *P, double *F, cudaStream_t st);

// The network (nrmg_net.cu) has these input and output channel counts, room for `pixels`
// pixels and runs on stream st.
bool net_fits(const ::nrmg_net *net, int cin, int cout, long long pixels, cudaStream_t st);

// Learned coarse-level correction (nrmg_net.cu): the scale s of the coarse change (device
// scalar) and the network input x [4 Hc Wc][NRMG_CORR_CIN] on the finest grid.
cudaError_t launch_corr_inputs(const double *coarse_before, const double *coarse_after, int Hc, int Wc,
                               const double *fine_fields, double lx, double ly, double Kn, double U, double *s_dev,
                               float *x, cudaStream_t st);
// f <- Grad(f + the increment of the ten learned fields U s y / NRMG_CORR_FIELD_SCALE) on every cell
// of L (nrmg_mixed.cu); y [ncell][10] FP32, s the device scalar above.
cudaError_t launch_field_correct(const Consts &K, const LevelDev &L, const float *y, const double *s_dev, double U,
                                 int grid, cudaStream_t st);

}  // namespace nrmg
