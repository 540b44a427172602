// nbody_internal.cuh -- internal declarations of libnbody (not installed).
//
// Data layout in device memory (all owned by a context):
//   x, v          FP64 SoA [3][npad]          positions / velocities
//   m             FP64 [npad]                 masses (pads have m = 0)
//   st            float4 [npad]               forward staging, pair layout:
//                   st[2p]   = (x_{2p}, x_{2p+1}, y_{2p}, y_{2p+1})
//                   st[2p+1] = (z_{2p}, z_{2p+1}, m_{2p}, m_{2p+1})
//                 coordinates are FP32 (x - c), c the FP64 recentring origin
//   vst           float4 [2*npad]             adjoint staging, pair layout:
//                   vst[4p]..vst[4p+1] as st, vst[4p+2] = -(lx, lx', ly, ly'),
//                   vst[4p+3] = (-lz, -lz', 0, 0), lambda the FP32 cotangent
//                   (stored negated)
//   part          FP64 [S][3][npad]           pair-kernel partial sums, one
//                                             slice per j-chunk, reduced in
//                                             fixed order by the consumer
// npad is n rounded up to a multiple of kPad; pad particles are staged at
// 1e18 with zero mass and zero cotangent, so their contribution is nil
// (exactly zero in the kernels that multiply by m_j, below 1e-33 relative
// in the equal-mass ones).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nbody.h"

namespace nb {

constexpr int kPad = 1024;

// Parameters read by the kernels from device memory, so that captured CUDA
// graphs stay valid when the parameters change.
struct DevParams {
  double G;
  double eps2;
  double dt;
  double nfw_GM, nfw_rs;
  double mn_GM, mn_a, mn_b;
  // bulge: G M_b, s = (3 - alpha)/2, 1/r_c^2, 1/r_c, 1/Gamma(s), Gamma(s - 1/2)
  double bulge_GM, bulge_s, bulge_irc2, bulge_irc, bulge_igs, bulge_gsh;
  uint32_t ext;
  uint32_t pad0;
  float eps2f;
  float pad1;
};

enum : int { kStatusNaN = 1, kStatusTimeout = 2 };

// columns of the adjoint's block accumulators: dL/d dt, sum_j m_j dL/dm_j,
// dL/dM_NFW, dL/dM_MN, dL/dr_s, dL/da_MN, dL/db_MN, dL/dM_bulge
constexpr int kAdjCols = 8;

// host: the bulge fields of DevParams from (M_b, alpha, r_c) and G
void set_bulge(DevParams& d, double G, double M, double alpha, double rc);

// ---- launch accounting ----
void count_launch(int k = 1);
long long thread_launches();  // launches counted by the calling thread
}  // namespace nb
struct nbody_mmd;
namespace nb {
// New target of the same size and bandwidths for an MMD evaluator, in place
// (device arrays); NBODY_ESTATE when it does not fit (mmd.cu).
int mmd_retarget(nbody_mmd* h, int64_t n, int64_t m, const double* tx, const double* tv,
                 const double* scale_or_null, int n_sigma, const double* sigma);
// Evaluator of `sets` clouds of n points, each against its own target of m
// points (ty, tv: device, 3 x sets m, target b in columns b m ..), in the
// caller's units (scale: 6 standard deviations); the targets' own terms are
// computed here (mmd.cu).  Destroy with nbody_mmd_destroy.
int mmd_create_multi(nbody_mmd** out, int64_t n, int64_t sets, int64_t m, const double* ty,
                     const double* tv, const double* scale, int n_sigma, const double* sigma,
                     cudaStream_t s);
// MMD^2 of every set against its target into loss (device, sets) and, when
// xbar and vbar (device, 3 x sets n) are given, its gradient; stream-ordered.
int mmd_eval_multi(nbody_mmd* h, const double* x, const double* v, double* loss, double* xbar,
                   double* vbar);

// ---- pair kernels (pair_force.cu, pair_vjp.cu) ----
enum PairVariant : int { kTile = 0, kWarp = 1 };

struct PairCfg {
  int variant;  // kTile: i-particles in registers, j-tiles in shared memory;
                // kWarp: lanes split j, warp-shuffle reduction (small n)
  int nt;       // threads per block
  int r;        // i-particles per thread (kTile) or per warp (kWarp)
  int S;        // number of j-chunks (grid.y); partial-sum slices
  bool eqm;     // equal masses: sums omit the mass, the consumer applies it
  int vjp_tile_pairs;  // j-pairs per shared-memory tile of the kernel
};

PairCfg choose_pair_cfg(int64_t npad, int sm_count, bool vjp, bool eqm);
int pair_blocks_per_sm(const PairCfg& c);
int vjp_blocks_per_sm(const PairCfg& c);
int vjp_tile_pairs();
bool pair_shape_supported(int variant, int nt, int r, bool vjp);
// the tile variant has an instance for this block shape and j-tile size
bool pair_tile_supported(int nt, int r, int tile_pairs, bool vjp);
int choose_chunks(const PairCfg& c, int64_t npad, int sm_count, int blocks_per_sm);

// Raw sums R_i = sum_j m_j (x_j - x_i) s_ij^-3 (no G; with cfg.eqm the
// common mass is left out too) into part[S][3][npad];
// with pot != NULL also P_i = sum_j m_j / s_ij (self term included) into
// pot[S][npad].
// The same (tile variant, S >= 2) with the S partial slices of every row
// tile summed by the tile's last-finishing block into fin [3][npad] (raw
// sums, ascending chunk order); ctr: one counter per row tile, zero between
// launches.  Other shapes fall back to launch_pair_accel (partials only).
cudaError_t launch_pair_accel_fin(const PairCfg& cfg, const float4* st, int64_t npad,
                                  float eps2, double* part, double* fin, unsigned* ctr,
                                  cudaStream_t s);
cudaError_t launch_pair_accel(const PairCfg& cfg, const float4* st,
                              int64_t npad, float eps2, double* part,
                              double* pot, cudaStream_t s);

// Raw sums Q_k = sum_j [s^-3 u - 3 s^-5 d (d.u)], u = m_j l_k - m_k l_j,
// d = x_j - x_k, into part[S][3][npad].  (J_pair^T l)_k = -G Q_k.  With
// cfg.eqm, u = l_k - l_j (the common mass is left out).
// With mpart != NULL also M_k = sum_j ((-l_j) . d) s^-3 into mpart[S][npad]
// (dL/dm_k = G sum over kicks of c M_k).
cudaError_t launch_pair_vjp(const PairCfg& cfg, const float4* vst,
                            int64_t npad, float eps2, double* part,
                            double* mpart, cudaStream_t s);
// The same with the slices of every row tile summed by its last-finishing
// block (tile variant, S >= 2; otherwise fin is ignored): Q into fin[0..2]
// [npad], M into fin[3][npad]; ctr as for launch_pair_accel_fin.
cudaError_t launch_pair_vjp_fin(const PairCfg& cfg, const float4* vst, int64_t npad,
                                float eps2, double* part, double* mpart, double* fin,
                                unsigned* ctr, cudaStream_t s);

// ---- per-particle kernels (update.cu) ----
cudaError_t launch_stage(const double* x, const double* m, const double* c,
                         int64_t n, int64_t npad, float4* st, cudaStream_t s);

struct UpdateArgs {
  const DevParams* P;
  int64_t n, npad;
  double* x;            // state, updated in place
  double* v;
  const double* part;   // pair partial sums (raw) or a final a_pair
  int S;                // slices in part
  int part_is_final;    // part holds G-scaled a_pair (one slice)
  double mscale;        // multiplies raw sums (the common mass, or 1)
  double* acc_out;      // receives a_pair (FSAL cache), may be NULL
  double kick;          // v += kick * a
  int drift;            // 1: x += dt * v after the kick, then restage
  const double* c_next; // recentring origin of the restaged positions
  float4* st;           // restaged positions
  double* cp_x;         // checkpoint slot (x, v before the kick, a_pair) or NULL
  double* cp_v;
  double* cp_a;
  double* tape_x;       // segment tape slot for this point (x, a_pair) or NULL
  double* tape_a;
  double* tape_vh;      // segment tape slot of the half-step velocity or NULL
  const double* aext;   // external acceleration at x [3][npad] (launch_field) or
                        // NULL: computed in the update
  int* status;
};
cudaError_t launch_update(const UpdateArgs& a, cudaStream_t s);
// FP64 external acceleration (G M included) of n particles into aext
// [3][npad]; runs beside the pair kernel of the same point
cudaError_t launch_field(const DevParams* P, const double* x, int64_t n, int64_t npad,
                         double* aext, cudaStream_t s);

// FP32 cotangent scaling of the reverse sweep: the cotangents staged for the
// pair VJP are multiplied by an exact power of two s = 2^-e chosen from the
// largest |lambda| of the previous point, so their FP32 copies never
// overflow or underflow while the FP64 cotangents grow or shrink (chaotic
// systems grow them exponentially).  lsc[0..1] holds the scale of the
// cotangents staged for points of even / odd index, lsc[2..3] (as unsigned
// 64-bit patterns of non-negative doubles) their running maxima.
constexpr int kLscDoubles = 4;

// lsc[2 + (p & 1)] = max |lam| over particles (atomic max of bit patterns)
cudaError_t launch_lam_absmax(const double* lam, int64_t n, int64_t npad,
                              double* lsc, int slot, cudaStream_t s);

// stages (x - c, m, s lam) with s derived from lsc[2 + slot]; writes s to
// lsc[slot]
cudaError_t launch_stage_vjp(const double* x, const double* m,
                             const double* lam, const double* c, int64_t n,
                             int64_t npad, float4* vst, double* lsc, int slot,
                             cudaStream_t s);

struct AdjointArgs {
  const DevParams* P;
  int64_t n, npad;
  double* xbar;          // running cotangents, updated in place
  double* vbar;
  const double* gpart;   // pair-VJP partial sums (raw)
  int S;
  double mscale;         // multiplies raw sums (the common mass, or 1)
  const double* xk;      // positions at this point
  const double* ak;      // a_pair at this point
  double ck;             // kick coefficient (dt/2 at the ends, dt inside)
  int drift;             // 1: also take the drift of the previous step
  const double* vh_prev; // v_{k-1/2}
  const double* x_prev;  // positions at the previous point (restaging)
  const double* c_prev;  // their recentring origin
  const double* m;
  float4* vst;           // restaged positions + new cotangent
  double* blk;           // [nblocks][kAdjCols] accumulators
  const double* mpart;   // mass-gradient partial sums [S][npad] or NULL
  double* mbar;          // running dL/dm [npad] (when mpart)
  double* lsc;           // cotangent scales (see kLscDoubles)
  int slot;              // parity of this point's index
  int* status;
  const double* ea;      // the external field's adjoint terms at this point,
                         // [kExtAdjCols][npad] from launch_ext_adjoint, or
                         // NULL: computed by the adjoint kernel itself
};
cudaError_t launch_adjoint(const AdjointArgs& a, cudaStream_t s);
// The external potential's adjoint terms at positions x with cotangents lam
// (x, lam [3][npad]) into ea [kExtAdjCols][npad]: H_ext(x) lam (3), the
// per-unit-mass products lam . a_NFW, lam . a_MN, lam . a_bulge (3) and the
// shape-parameter terms (3), the same values the adjoint kernel computes
// when it is given no ea (update.cu).
constexpr int kExtAdjCols = 9;
cudaError_t launch_ext_adjoint(const DevParams* P, const double* x, const double* lam,
                               int64_t n, int64_t npad, double* ea, cudaStream_t s);
int adjoint_blocks(int64_t n);

// out[0..1] = min and max of m[0..n)
cudaError_t launch_minmax(const double* m, int64_t n, double* out, cudaStream_t s);
cudaError_t launch_ext_accel(const DevParams& P, const double* x, int64_t n, double* acc,
                             cudaStream_t s);

cudaError_t launch_reduce_rows(const double* blk, int nblk, int ncol,
                               double* out, cudaStream_t s);

cudaError_t launch_guide(const DevParams* P, const double* g0, int64_t n_steps,
                         double* centers, double* g_out, cudaStream_t s);

cudaError_t launch_energy(const DevParams* P, const double* x,
                          const double* v, const double* m, int64_t n,
                          const double* pot_part, int S, int64_t npad,
                          double* blk, int nblk, cudaStream_t s);
int energy_blocks(int64_t n);

cudaError_t launch_reduce_partials(const double* part, int S, int64_t npad,
                                   int64_t n, double G, double* acc,
                                   cudaStream_t s);

// ---- batched ensemble (batch.cu) ----
struct Batch;
int batch_create(Batch** out, int n_sims, const int64_t* offsets,
                 const nbody_params* p, cudaStream_t user, int sm_count);
void batch_destroy(Batch* b);
int batch_set_params(Batch* b, const nbody_params* p);
int batch_set_state(Batch* b, const double* x, const double* v, const double* m);
int batch_get_state(Batch* b, double* x, double* v);
int batch_integrate(Batch* b, int64_t n_steps);
// reverse sweep of the last recorded run (every simulation's
// checkpoint_every > 0); cotangents and results in the caller's layout,
// theta_bar [n_sims][kAdjCols] or NULL
int batch_vjp(Batch* b, const double* xbar, const double* vbar, double* x0bar, double* v0bar,
              double* theta_bar);
// whether batch_vjp forms the shape-parameter gradients (default yes; the
// batched pipeline, which needs the masses only, turns them off)
void batch_set_vjp_shape(Batch* b, bool on);
// clears the batch's sticky NaN status (the batched pipeline reports failed
// members itself)
int batch_clear_status(Batch* b);
// the batch behind a batch context (nbody_api.cu)
Batch* context_batch(nbody_ctx* c);
int batch_status(Batch* b);
int batch_autotune(Batch* b, int64_t probe_steps, int* best, double* ms);
int batch_set_tuning(Batch* b, int k);
int batch_tuning(Batch* b);

}  // namespace nb
