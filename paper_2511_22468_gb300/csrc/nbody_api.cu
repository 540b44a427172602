// nbody_api.cu -- the C ABI of libnbody (declared in include/nbody.h): the
// context, its device memory, the forward driver (kick-drift-kick with
// checkpoints and tape) and the reverse sweep (discrete adjoint with
// segment recomputation).
//
// Forward (Velocity-Verlet, paper Sec. 2.2.1), points k = 0..n:
//   pair pass at x_k (FP32, pair_force.cu) -> update kernel: a = a_pair +
//   a_ext(x_k); v += c_k a (c_k = dt/2 at k = 0 and k = n, dt between: the
//   closing and opening half kicks at one point merged); if k < n:
//   x += dt v and restage x_{k+1} for the next pair pass.
// The acceleration at the final point is kept (first-same-as-last) and
// reused by the next call.
//
// Tape (reverse-mode gradients, Sec. 2): checkpoint c at point cK stores
// (x_k, v before the kick at k, a_pair(x_k)); the end point is one more
// checkpoint.  A segment buffer holds, for the K points of one segment,
// x_k, a_pair(x_k) and the half-step velocities.  The reverse sweep walks
// the segments backward, recomputing each from its checkpoint (K - 1 pair
// passes: both end accelerations are in the checkpoints), and at every
// point k runs the pair VJP and the adjoint update.  Every kernel sums in a
// fixed order, so the recomputation reproduces the forward pass bit for bit.
#include <cuda_runtime.h>

#include <algorithm>

#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "nbody_internal.cuh"

namespace nb {
static std::atomic<long long> g_launches{0};
// this thread's launches: a graph capture counts its nodes from it, so that
// other threads' launches in the meantime are not taken for recorded ones
static thread_local long long t_launches = 0;
void count_launch(int k) {
  g_launches.fetch_add(k, std::memory_order_relaxed);
  t_launches += k;
}
long long thread_launches() { return t_launches; }
}  // namespace nb

using nb::DevParams;

struct nbody_ctx {
  int dev = 0;
  int sm_count = 0;
  int64_t n = 0, npad = 0;
  cudaStream_t stream = nullptr;
  nbody_params p{};
  DevParams hp{};
  DevParams* dp = nullptr;

  double* x = nullptr;  // [3][npad]
  double* v = nullptr;
  double* m = nullptr;  // [npad]
  double* acc = nullptr;  // FSAL a_pair cache [3][npad]
  bool acc_valid = false;
  float4* st = nullptr;   // [npad]
  float4* vst = nullptr;  // [2*npad]
  double* part = nullptr; // [Smax][3][npad]
  double* pot = nullptr;  // [Sf][npad]
  double* fin = nullptr;  // pair (or VJP) sums with the slices summed [4][npad]
  unsigned* pctr = nullptr;  // finished-chunk counters per row tile [npad/128]
  int fin_mode = -1;  // forward slices summed in the pair kernel: 1 yes, 0 no,
                      // -1 by chunk count (S >= 8)
  int vfin_mode = -1;  // the same for the VJP kernel
  int Smax = 0;
  nb::PairCfg fcfg{}, vcfg{};
  double m_eq = 1.0;  // the common mass when fcfg.eqm / vcfg.eqm
  bool shape_fixed[2] = {false, false};  // launch shape set by the caller

  double* guide = nullptr;       // [6] current guide (x, v)
  double* fixed_center = nullptr;  // [3]
  double* centers = nullptr;     // [(cap+1)*3]
  int64_t centers_cap = 0;

  // tape
  int64_t tape_steps = 0;
  int64_t K = 0, nseg = 0;
  bool last_seg_valid = false;
  double* cp = nullptr;  // [(nseg+1)][9][npad]
  int64_t cp_cap = 0;    // checkpoints allocated
  double* seg = nullptr; // [3K][3][npad]
  int64_t seg_cap = 0;   // K allocated
  double* xw = nullptr;  // recompute work state [3][npad] x2
  double* vw = nullptr;
  // small systems: the reverse sweep of a segment runs beside the
  // recomputation of the segment before it (stream rs2, the second segment
  // buffer, its own pair-kernel scratch), so that two kernels share the SMs
  double* seg2 = nullptr;  // [3K][3][npad]
  int64_t seg2_cap = 0;
  float4* st2 = nullptr;
  double* part2 = nullptr;
  double* fin2 = nullptr;
  unsigned* pctr2 = nullptr;
  cudaStream_t rs2 = nullptr;
  cudaEvent_t ev_rfork = nullptr, ev_rready = nullptr;

  // adjoint
  double* xbar = nullptr;
  double* vbar = nullptr;
  double* blk = nullptr;  // [nblk][max(kAdjCols, 6)]
  double* red = nullptr;  // [8]
  double* lsc = nullptr;  // cotangent scales [kLscDoubles]
  double* mpart = nullptr;  // mass-gradient partial sums [Smax][npad], lazily
  // the FP64 external field of a point runs on a side stream beside that
  // point's pair kernel (different pipes), joined before the update
  double* aext = nullptr;   // [3][npad]
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // likewise the FP64 external-field terms of the adjoint at a point run on
  // a second side stream beside that point's pair VJP (allocated with the
  // tape when the context has an external potential)
  double* ea = nullptr;     // [kExtAdjCols][npad]
  cudaStream_t aside = nullptr;
  cudaEvent_t ev_afork = nullptr, ev_ajoin = nullptr;
  double* mbar = nullptr;   // dL/dm [npad], lazily
  bool want_mbar = false;   // the sweep being recorded accumulates dL/dm
  double pot_bar[6] = {0, 0, 0, 0, 0, 0};  // last sweep's potential-parameter gradient
  bool have_grad = false;
  int nblk = 0;
  int* status = nullptr;

  // captured step loops: forward and reverse sweeps replayed as CUDA graphs
  struct GraphEntry {
    uint64_t key[12];
    cudaGraphExec_t exec;
    int nodes;
    uint64_t stamp;
  };
  std::vector<GraphEntry> graphs;
  uint64_t graph_stamp = 0;
  cudaStream_t gs = nullptr;
  cudaEvent_t gev_in = nullptr, gev_out = nullptr;

  // batched ensemble (all other buffers unused when set)
  nb::Batch* batch = nullptr;
  int n_sims = 0;

  // per-kernel event timing
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[NBODY_NKCLASS];
  size_t ev_used[NBODY_NKCLASS] = {};
};

namespace nb {
Batch* context_batch(nbody_ctx* c) { return c ? c->batch : nullptr; }
}  // namespace nb

namespace {

#define CK(call)                              \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return NBODY_ECUDA; \
  } while (0)

int check_params(const nbody_params* p) {
  if (!p) return NBODY_EINVAL;
  if (!(p->eps > 0.0) || !std::isfinite(p->eps)) return NBODY_EINVAL;
  if (!std::isfinite(p->G) || !std::isfinite(p->dt)) return NBODY_EINVAL;
  if (p->checkpoint_every < 0) return NBODY_EINVAL;
  if (p->ext_flags & ~(NBODY_EXT_NFW | NBODY_EXT_MN | NBODY_EXT_BULGE)) return NBODY_EINVAL;
  if (p->center_mode > NBODY_CENTER_GUIDE) return NBODY_EINVAL;
  if (p->tape_mode > NBODY_TAPE_LEAN) return NBODY_EINVAL;
  if (p->reserved != 0) return NBODY_EINVAL;
  if ((p->ext_flags & NBODY_EXT_NFW) && !(p->nfw_rs > 0.0)) return NBODY_EINVAL;
  if ((p->ext_flags & NBODY_EXT_MN) && !(p->mn_b >= 0.0 && p->mn_a >= 0.0))
    return NBODY_EINVAL;
  if ((p->ext_flags & NBODY_EXT_BULGE) &&
      !(std::isfinite(p->bulge_M) && p->bulge_alpha >= 0.0 && p->bulge_alpha < 2.0 &&
        p->bulge_rc > 0.0 && std::isfinite(p->bulge_rc)))
    return NBODY_EINVAL;
  return NBODY_OK;
}

DevParams to_dev(const nbody_params& p) {
  DevParams d{};
  d.G = p.G;
  d.eps2 = p.eps * p.eps;
  d.dt = p.dt;
  d.ext = p.ext_flags;
  d.nfw_GM = (p.ext_flags & NBODY_EXT_NFW) ? p.G * p.nfw_M : 0.0;
  d.nfw_rs = (p.ext_flags & NBODY_EXT_NFW) ? p.nfw_rs : 1.0;
  d.mn_GM = (p.ext_flags & NBODY_EXT_MN) ? p.G * p.mn_M : 0.0;
  d.mn_a = p.mn_a;
  d.mn_b = p.mn_b;
  d.eps2f = (float)(p.eps * p.eps);
  if (p.ext_flags & NBODY_EXT_BULGE) nb::set_bulge(d, p.G, p.bulge_M, p.bulge_alpha, p.bulge_rc);
  return d;
}

template <class T>
int dalloc(T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc((void**)ptr, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return NBODY_ENOMEM;
  }
  return NBODY_OK;
}

template <class T>
void dfree(T*& ptr) {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
}

int upload_params(nbody_ctx* c) {
  c->hp = to_dev(c->p);
  CK(cudaMemcpyAsync(c->dp, &c->hp, sizeof(DevParams), cudaMemcpyHostToDevice,
                     c->stream));
  double g[6] = {c->p.center[0], c->p.center[1], c->p.center[2],
                 c->p.center_vel[0], c->p.center_vel[1], c->p.center_vel[2]};
  CK(cudaMemcpyAsync(c->fixed_center, c->p.center, 3 * sizeof(double),
                     cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->guide, g, 6 * sizeof(double), cudaMemcpyHostToDevice,
                     c->stream));
  // pageable sources: make the copies complete before the host arrays die
  CK(cudaStreamSynchronize(c->stream));
  return NBODY_OK;
}

// Launch through f(), bracketed by two events on the context stream when
// timing is enabled.
template <class F>
cudaError_t timed(nbody_ctx* c, int cls, F&& f) {
  if (!c->timing) return f();
  auto& pool = c->ev[cls];
  const size_t k = c->ev_used[cls];
  if (k == pool.size()) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
      cudaEventDestroy(a);
      return e;
    }
    pool.emplace_back(a, b);
  }
  cudaError_t e = cudaEventRecord(pool[k].first, c->stream);
  if (e != cudaSuccess) return e;
  e = f();
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(pool[k].second, c->stream);
  c->ev_used[cls] = k + 1;
  return e;
}

void drop_graphs(nbody_ctx* c) {
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

// Step loops of small systems are launch-bound: they are captured once per
// configuration (key) on an internal stream and replayed.  Every kernel reads
// its parameters from device memory, so a replay stays valid when the
// parameters change; anything else the launches bake in is part of the key,
// and buffer reallocation drops the cache.
bool graph_eligible(const nbody_ctx* c, int64_t n_steps) {
  return !c->timing && c->npad <= 262144 && n_steps >= 4;
}

// the overlapped reverse sweep: small systems, whose kernels leave SMs idle,
// and not under per-kernel event timing (events on one stream)
bool use_overlap(const nbody_ctx* c) {
  return !c->timing && c->npad < 65536 && c->rs2 != nullptr;
}

template <class F>
int run_graph(nbody_ctx* c, const uint64_t (&key)[12], F record) {
  if (!c->gs) {
    if (cudaStreamCreateWithFlags(&c->gs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->gev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->gev_out, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return NBODY_ECUDA;
    }
  }
  nbody_ctx::GraphEntry* hit = nullptr;
  for (auto& g : c->graphs)
    if (std::memcmp(g.key, key, sizeof(key)) == 0) hit = &g;
  if (!hit) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamSynchronize(c->gs));
    CK(cudaStreamBeginCapture(c->gs, cudaStreamCaptureModeThreadLocal));
    const long long before = nb::thread_launches();
    const int rc = record(c->gs);
    const int nodes = (int)(nb::thread_launches() - before);
    nb::count_launch(-nodes);  // recorded, not launched
    const cudaError_t e = cudaStreamEndCapture(c->gs, &graph);
    if (rc || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc ? rc : NBODY_ECUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      cudaGetLastError();
      return NBODY_ECUDA;
    }
    if (c->graphs.size() >= 4) {  // evict the least recently used
      size_t old = 0;
      for (size_t i = 1; i < c->graphs.size(); ++i)
        if (c->graphs[i].stamp < c->graphs[old].stamp) old = i;
      cudaGraphExecDestroy(c->graphs[old].exec);
      c->graphs.erase(c->graphs.begin() + old);
    }
    nbody_ctx::GraphEntry g;
    std::memcpy(g.key, key, sizeof(key));
    g.exec = exec;
    g.nodes = nodes;
    g.stamp = 0;
    c->graphs.push_back(g);
    hit = &c->graphs.back();
  }
  hit->stamp = ++c->graph_stamp;
  CK(cudaEventRecord(c->gev_in, c->stream));
  CK(cudaStreamWaitEvent(c->gs, c->gev_in, 0));
  CK(cudaGraphLaunch(hit->exec, c->gs));
  CK(cudaEventRecord(c->gev_out, c->gs));
  CK(cudaStreamWaitEvent(c->stream, c->gev_out, 0));
  nb::count_launch(hit->nodes);
  return NBODY_OK;
}

uint64_t bits(double v) {
  uint64_t u;
  std::memcpy(&u, &v, sizeof(u));
  return u;
}

uint64_t cfg_word(const nb::PairCfg& f) {
  return (uint64_t)f.variant | ((uint64_t)f.nt << 4) | ((uint64_t)f.r << 16) |
         ((uint64_t)f.S << 24) | ((uint64_t)f.eqm << 40) |
         ((uint64_t)(f.vjp_tile_pairs >> 7) << 41);
}

// centre of point k of the current call
const double* center_at(nbody_ctx* c, int64_t k) {
  if (c->p.center_mode == NBODY_CENTER_GUIDE) return c->centers + 3 * k;
  return c->fixed_center;
}

int ensure_centers(nbody_ctx* c, int64_t n_steps) {
  if (c->centers_cap >= n_steps && c->centers) return NBODY_OK;
  drop_graphs(c);
  dfree(c->centers);
  c->centers_cap = 0;
  int rc = dalloc(&c->centers, (size_t)(n_steps + 1) * 3);
  if (rc) return rc;
  c->centers_cap = n_steps;
  return NBODY_OK;
}

// The adjoint's external-field terms run beside the pair VJP for systems
// whose VJP launch is long enough to hide them (measured on GB300: at
// npad = 3072 the 18 us VJP cannot cover the FP64 terms and the sweep
// slows, at 10240 it gains 13 %); large systems keep them in the adjoint
// kernel, where they are a small fraction of a point.
bool ext_adjoint_beside(const nbody_ctx* c) { return c->npad >= 8192 && c->npad < 65536; }

int ensure_tape(nbody_ctx* c, int64_t nseg, int64_t K) {
  const size_t slot = (size_t)3 * c->npad;
  if (c->cp_cap < nseg + 1 || !c->cp) {
    drop_graphs(c);
    dfree(c->cp);
    c->cp_cap = 0;
    int rc = dalloc(&c->cp, (size_t)(nseg + 1) * 3 * slot);
    if (rc) return rc;
    c->cp_cap = nseg + 1;
  }
  if (c->seg_cap < K || !c->seg) {
    drop_graphs(c);
    dfree(c->seg);
    c->seg_cap = 0;
    int rc = dalloc(&c->seg, (size_t)3 * K * slot);
    if (rc) return rc;
    c->seg_cap = K;
  }
  if (!c->xw) {
    drop_graphs(c);
    int rc = dalloc(&c->xw, slot);
    if (rc) return rc;
    rc = dalloc(&c->vw, slot);
    if (rc) return rc;
  }
  if (c->p.ext_flags && !c->ea && ext_adjoint_beside(c)) {  // field terms beside the VJP
    drop_graphs(c);
    int rc = dalloc(&c->ea, (size_t)nb::kExtAdjCols * c->npad);
    if (rc) return rc;
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if ((!c->ev_afork &&
         cudaEventCreateWithFlags(&c->ev_afork, cudaEventDisableTiming) != cudaSuccess) ||
        (!c->ev_ajoin &&
         cudaEventCreateWithFlags(&c->ev_ajoin, cudaEventDisableTiming) != cudaSuccess) ||
        cudaStreamCreateWithPriority(&c->aside, cudaStreamNonBlocking, prio_hi) != cudaSuccess) {
      cudaGetLastError();
      c->aside = nullptr;
      dfree(c->ea);
      return NBODY_ECUDA;
    }
  }
  if (c->npad < 65536 && nseg >= 2) {  // the overlapped sweep's second buffer and scratch
    if (c->seg2_cap < K || !c->seg2) {
      drop_graphs(c);
      dfree(c->seg2);
      c->seg2_cap = 0;
      int rc = dalloc(&c->seg2, (size_t)3 * K * slot);
      if (rc) return rc;
      c->seg2_cap = K;
    }
    if (!c->rs2) {
      drop_graphs(c);
      const size_t np = (size_t)c->npad;
      int rc = NBODY_OK;
      if (!c->st2) rc = dalloc(&c->st2, np);
      if (!rc && !c->part2) rc = dalloc(&c->part2, (size_t)c->Smax * 3 * np);
      if (!rc && !c->fin2) rc = dalloc(&c->fin2, 4 * np);
      if (!rc && !c->pctr2) {
        rc = dalloc(&c->pctr2, np / 128);
        if (!rc && cudaMemsetAsync(c->pctr2, 0, (np / 128) * sizeof(unsigned), c->stream) !=
                       cudaSuccess) {
          cudaGetLastError();
          dfree(c->pctr2);
          rc = NBODY_ECUDA;
        }
      }
      if (rc) return rc;
      if ((!c->ev_rfork &&
           cudaEventCreateWithFlags(&c->ev_rfork, cudaEventDisableTiming) != cudaSuccess) ||
          (!c->ev_rready &&
           cudaEventCreateWithFlags(&c->ev_rready, cudaEventDisableTiming) != cudaSuccess) ||
          cudaStreamCreateWithFlags(&c->rs2, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        c->rs2 = nullptr;
        return NBODY_ECUDA;
      }
    }
  }
  return NBODY_OK;
}

struct Tape {
  nbody_ctx* c;
  size_t slot;
  double* seg = nullptr;  // segment buffer (the context's first when null)
  double* base() const { return seg ? seg : c->seg; }
  double* cpx(int64_t i) const { return c->cp + (size_t)i * 3 * slot; }
  double* cpv(int64_t i) const { return cpx(i) + slot; }
  double* cpa(int64_t i) const { return cpx(i) + 2 * slot; }
  double* sx(int64_t j) const { return base() + (size_t)j * slot; }
  double* sa(int64_t j) const { return base() + (size_t)(c->K + j) * slot; }
  double* svh(int64_t j) const {  // j = 1..K
    return base() + (size_t)(2 * c->K + j - 1) * slot;
  }
};

// the pair kernel's staging and sums used by a forward run or recomputation
struct PairScratch {
  float4* st;
  double* part;
  double* fin;
  unsigned* pctr;
};
PairScratch primary_scratch(nbody_ctx* c) { return {c->st, c->part, c->fin, c->pctr}; }
PairScratch second_scratch(nbody_ctx* c) { return {c->st2, c->part2, c->fin2, c->pctr2}; }

nb::UpdateArgs base_update(nbody_ctx* c, double* x, double* v, const PairScratch& sc) {
  nb::UpdateArgs a{};
  a.P = c->dp;
  a.n = c->n;
  a.npad = c->npad;
  a.x = x;
  a.v = v;
  a.part = sc.part;
  a.S = c->fcfg.S;
  a.part_is_final = 0;
  a.mscale = c->fcfg.eqm ? c->m_eq : 1.0;
  a.st = sc.st;
  a.status = c->status;
  return a;
}

nb::UpdateArgs base_update(nbody_ctx* c, double* x, double* v) {
  return base_update(c, x, v, primary_scratch(c));
}

// The external field of the point x is computed on the side stream while
// stream s runs that point's pair kernel; the update waits for both.
// Under per-kernel timing the field runs on stream s itself, so that its
// events time the kernel rather than its wait for SMs beside the pair kernel.
int fork_field(nbody_ctx* c, const double* x, cudaStream_t s) {
  if (!c->p.ext_flags || !c->side) return NBODY_OK;
  if (c->timing) {
    CK(timed(c, NBODY_KCLASS_FIELD,
             [&] { return nb::launch_field(c->dp, x, c->n, c->npad, c->aext, s); }));
    return NBODY_OK;
  }
  CK(cudaEventRecord(c->ev_fork, s));
  CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
  CK(nb::launch_field(c->dp, x, c->n, c->npad, c->aext, c->side));
  CK(cudaEventRecord(c->ev_join, c->side));
  return NBODY_OK;
}

int join_field(nbody_ctx* c, cudaStream_t s, nb::UpdateArgs& a) {
  if (!c->p.ext_flags || !c->side) return NBODY_OK;
  if (!c->timing) CK(cudaStreamWaitEvent(s, c->ev_join, 0));
  a.aext = c->aext;
  return NBODY_OK;
}

// The pair kernel of one forward point; with the tile kernel split into
// S >= 2 j-chunks its last block per row tile sums the slices, and the
// update reads that one slice (same sums, same order).
bool use_fin(const nb::PairCfg& f, int mode) {
  if (f.variant != nb::kTile || f.S < 2) return false;
  return mode < 0 ? f.S >= 8 : mode == 1;
}

int pair_forward(nbody_ctx* c, nb::UpdateArgs& a, cudaStream_t s, const PairScratch& sc) {
  const bool fin = use_fin(c->fcfg, c->fin_mode);
  CK(timed(c, NBODY_KCLASS_PAIR, [&] {
    return fin ? nb::launch_pair_accel_fin(c->fcfg, sc.st, c->npad, c->hp.eps2f, sc.part,
                                           sc.fin, sc.pctr, s)
               : nb::launch_pair_accel(c->fcfg, sc.st, c->npad, c->hp.eps2f, sc.part,
                                       nullptr, s);
  }));
  if (fin) {
    a.part = sc.fin;
    a.S = 1;
  }
  return NBODY_OK;
}

int pair_forward(nbody_ctx* c, nb::UpdateArgs& a, cudaStream_t s) {
  return pair_forward(c, a, s, primary_scratch(c));
}

// The launches of a forward run over points 0..n_steps (on stream s).
int record_forward(nbody_ctx* c, int64_t n_steps, bool with_tape, cudaStream_t s) {
  if (c->p.center_mode == NBODY_CENTER_GUIDE)
    CK(nb::launch_guide(c->dp, c->guide, n_steps, c->centers, c->guide, s));
  const int64_t K = with_tape ? c->K : 0;
  const int64_t nseg = with_tape ? c->nseg : 0;
  const int64_t ls = nseg - 1;
  Tape T{c, (size_t)3 * c->npad};
  const bool keep_last = with_tape && c->p.tape_mode == NBODY_TAPE_KEEP_LAST;
  for (int64_t k = 0; k <= n_steps; ++k) {
    nb::UpdateArgs a = base_update(c, c->x, c->v);
    if (k == 0 && c->acc_valid) {
      a.part = c->acc;
      a.S = 1;
      a.part_is_final = 1;
    } else {
      if (k == 0)
        CK(nb::launch_stage(c->x, c->m, center_at(c, 0), c->n, c->npad, c->st, s));
      if (int r_ = fork_field(c, c->x, s)) return r_;
      if (int r_ = pair_forward(c, a, s)) return r_;
      if (int r_ = join_field(c, s, a)) return r_;
    }
    a.acc_out = (k == n_steps) ? c->acc : nullptr;
    a.kick = (k == 0 || k == n_steps) ? 0.5 : 1.0;
    a.drift = k < n_steps;
    a.c_next = a.drift ? center_at(c, k + 1) : nullptr;
    if (with_tape) {
      if (k % K == 0 || k == n_steps) {
        const int64_t ci = (k == n_steps) ? nseg : k / K;
        a.cp_x = T.cpx(ci);
        a.cp_v = T.cpv(ci);
        a.cp_a = T.cpa(ci);
      }
      if (keep_last && k >= ls * K && k < n_steps) {
        const int64_t j = k - ls * K;
        a.tape_x = T.sx(j);
        a.tape_a = T.sa(j);
        a.tape_vh = T.svh(j + 1);
      }
    }
    CK(timed(c, NBODY_KCLASS_UPDATE, [&] { return nb::launch_update(a, s); }));
  }
  return NBODY_OK;
}

// Forward over points 0..n_steps from the live state; with_tape records
// checkpoints (and the last segment unless the tape is lean).
int run_forward(nbody_ctx* c, int64_t n_steps, bool with_tape) {
  int rc = ensure_centers(c, n_steps);
  if (rc) return rc;
  const int64_t K = with_tape ? c->p.checkpoint_every : 0;
  if (with_tape) {
    const int64_t nseg = (n_steps + K - 1) / K;
    rc = ensure_tape(c, nseg, K);
    if (rc) return rc;
    c->K = K;
    c->nseg = nseg;
  }
  const bool keep_last = with_tape && c->p.tape_mode == NBODY_TAPE_KEEP_LAST;
  if (graph_eligible(c, n_steps)) {
    const uint64_t key[12] = {1, (uint64_t)n_steps, (uint64_t)with_tape, (uint64_t)K,
                              (uint64_t)c->p.tape_mode, (uint64_t)c->acc_valid,
                              (uint64_t)c->p.center_mode, cfg_word(c->fcfg), bits(c->m_eq),
                              (uint64_t)use_fin(c->fcfg, c->fin_mode), 0, 0};
    rc = run_graph(c, key, [&](cudaStream_t gs) { return record_forward(c, n_steps, with_tape, gs); });
  } else {
    rc = record_forward(c, n_steps, with_tape, c->stream);
  }
  if (rc) return rc;
  c->acc_valid = true;
  if (with_tape) {
    c->tape_steps = n_steps;
    c->last_seg_valid = keep_last;
  } else {
    c->tape_steps = 0;
    c->last_seg_valid = false;
  }
  return NBODY_OK;
}

// Recompute segment sg from its checkpoint into the segment buffer seg
// (the context's first when null), with the pair-kernel scratch sc.
int recompute_segment(nbody_ctx* c, int64_t sg, cudaStream_t s, const PairScratch& sc,
                      double* seg) {
  Tape T{c, (size_t)3 * c->npad, seg};
  const int64_t K = c->K, n = c->tape_steps;
  const int64_t k0 = sg * K;
  const int64_t Ks = (k0 + K <= n) ? K : n - k0;
  const size_t bytes = (size_t)3 * c->npad * sizeof(double);
  CK(cudaMemcpyAsync(c->xw, T.cpx(sg), bytes, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(c->vw, T.cpv(sg), bytes, cudaMemcpyDeviceToDevice, s));
  for (int64_t j = 0; j < Ks; ++j) {
    const int64_t k = k0 + j;
    nb::UpdateArgs a = base_update(c, c->xw, c->vw, sc);
    if (j == 0) {
      a.part = T.cpa(sg);
      a.S = 1;
      a.part_is_final = 1;
    } else {
      if (int r_ = fork_field(c, c->xw, s)) return r_;
      if (int r_ = pair_forward(c, a, s, sc)) return r_;
      if (int r_ = join_field(c, s, a)) return r_;
    }
    a.kick = (k == 0) ? 0.5 : 1.0;
    a.drift = 1;
    a.c_next = center_at(c, k + 1);
    a.tape_x = T.sx(j);
    a.tape_a = T.sa(j);
    a.tape_vh = T.svh(j + 1);
    CK(timed(c, NBODY_KCLASS_UPDATE, [&] { return nb::launch_update(a, s); }));
  }
  return NBODY_OK;
}

int copy_in(double* dst, const double* src, size_t count, cudaStream_t s) {
  CK(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDefault, s));
  return NBODY_OK;
}

// copy a [3][n] caller array into a [3][npad] device array
int copy_in3(nbody_ctx* c, double* dst, const double* src) {
  for (int d = 0; d < 3; ++d) {
    int rc = copy_in(dst + (size_t)d * c->npad, src + (size_t)d * c->n,
                     (size_t)c->n, c->stream);
    if (rc) return rc;
  }
  return NBODY_OK;
}

int copy_out3(nbody_ctx* c, double* dst, const double* src) {
  for (int d = 0; d < 3; ++d)
    CK(cudaMemcpyAsync(dst + (size_t)d * c->n, src + (size_t)d * c->npad,
                       (size_t)c->n * sizeof(double), cudaMemcpyDefault,
                       c->stream));
  return NBODY_OK;
}

void free_all(nbody_ctx* c) {
  if (c->side) cudaStreamDestroy(c->side);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  c->side = nullptr;
  c->ev_fork = c->ev_join = nullptr;
  dfree(c->aext);
  if (c->aside) cudaStreamDestroy(c->aside);
  if (c->ev_afork) cudaEventDestroy(c->ev_afork);
  if (c->ev_ajoin) cudaEventDestroy(c->ev_ajoin);
  c->aside = nullptr;
  c->ev_afork = c->ev_ajoin = nullptr;
  dfree(c->ea);
  for (auto& pool : c->ev)
    for (auto& pr : pool) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  dfree(c->dp);
  dfree(c->x);
  dfree(c->v);
  dfree(c->m);
  dfree(c->acc);
  dfree(c->st);
  dfree(c->vst);
  dfree(c->part);
  dfree(c->pot);
  dfree(c->fin);
  dfree(c->pctr);
  dfree(c->guide);
  dfree(c->fixed_center);
  dfree(c->centers);
  dfree(c->cp);
  dfree(c->seg);
  dfree(c->seg2);
  dfree(c->st2);
  dfree(c->part2);
  dfree(c->fin2);
  dfree(c->pctr2);
  if (c->rs2) cudaStreamDestroy(c->rs2);
  if (c->ev_rfork) cudaEventDestroy(c->ev_rfork);
  if (c->ev_rready) cudaEventDestroy(c->ev_rready);
  c->rs2 = nullptr;
  c->ev_rfork = c->ev_rready = nullptr;
  dfree(c->xw);
  dfree(c->vw);
  dfree(c->xbar);
  dfree(c->vbar);
  dfree(c->blk);
  dfree(c->red);
  dfree(c->lsc);
  dfree(c->mpart);
  dfree(c->mbar);
  dfree(c->status);
}

int check_device(int* dev, int* sms) {
  if (cudaGetDevice(dev) != cudaSuccess) {
    cudaGetLastError();
    return NBODY_ENODEV;
  }
  int maj = 0, min = 0;
  if (cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, *dev) ||
      cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, *dev) ||
      cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, *dev)) {
    cudaGetLastError();
    return NBODY_ENODEV;
  }
  if (maj != 10 || min != 3) return NBODY_ENODEV;
  return NBODY_OK;
}

}  // namespace

extern "C" {

const char* nbody_strerror(int code) {
  switch (code) {
    case NBODY_OK: return "ok";
    case NBODY_EINVAL: return "invalid argument";
    case NBODY_ENOMEM: return "out of memory";
    case NBODY_ECUDA: return "CUDA runtime error";
    case NBODY_ETIMEOUT: return "bounded device wait expired";
    case NBODY_ENAN: return "non-finite value in the state";
    case NBODY_ESTATE: return "call out of order (no tape recorded)";
    case NBODY_ENODEV: return "no sm_103a device";
    case NBODY_ESIZE: return "size exceeds the fixed buffer of this call";
    default: return "unknown status";
  }
}

int64_t nbody_launch_count(void) { return nb::g_launches.load(); }

int nbody_create(nbody_ctx** out, int64_t n, const nbody_params* p,
                 void* cuda_stream) {
  if (!out) return NBODY_EINVAL;
  *out = nullptr;
  if (n < 1) return NBODY_EINVAL;
  int rc = check_params(p);
  if (rc) return rc;
  int dev = 0, sms = 0;
  rc = check_device(&dev, &sms);
  if (rc) return rc;
  nbody_ctx* c = new (std::nothrow) nbody_ctx();
  if (!c) return NBODY_ENOMEM;
  c->dev = dev;
  c->sm_count = sms;
  c->n = n;
  c->npad = ((n + nb::kPad - 1) / nb::kPad) * nb::kPad;
  c->stream = (cudaStream_t)cuda_stream;
  c->p = *p;
  c->fcfg = nb::choose_pair_cfg(c->npad, sms, false, false);
  c->vcfg = nb::choose_pair_cfg(c->npad, sms, true, false);
  c->Smax = 32;  // the largest chunk count choose_chunks picks
  const size_t np = (size_t)c->npad;
  c->nblk = nb::adjoint_blocks(n);
  if ((rc = dalloc(&c->dp, 1)) || (rc = dalloc(&c->x, 3 * np)) ||
      (rc = dalloc(&c->v, 3 * np)) || (rc = dalloc(&c->m, np)) ||
      (rc = dalloc(&c->acc, 3 * np)) || (rc = dalloc(&c->st, np)) ||
      (rc = dalloc(&c->vst, 2 * np)) ||
      (rc = dalloc(&c->part, (size_t)c->Smax * 3 * np)) ||
      (rc = dalloc(&c->pot, (size_t)c->Smax * np)) ||
      (rc = dalloc(&c->guide, 6)) || (rc = dalloc(&c->fixed_center, 3)) ||
      (rc = dalloc(&c->xbar, 3 * np)) || (rc = dalloc(&c->vbar, 3 * np)) ||
      (rc = dalloc(&c->blk, (size_t)c->nblk * std::max(nb::kAdjCols, 6))) || (rc = dalloc(&c->red, 8)) || (rc = dalloc(&c->lsc, nb::kLscDoubles)) ||
      (rc = dalloc(&c->status, 1)) || (rc = dalloc(&c->aext, 3 * np)) ||
      (rc = dalloc(&c->fin, 4 * np)) || (rc = dalloc(&c->pctr, np / 128))) {
    free_all(c);
    delete c;
    return rc;
  }
  // the side stream takes the highest priority, so that the small field
  // kernel's blocks are placed before the pair kernel fills the SMs
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    free_all(c);
    delete c;
    return NBODY_ECUDA;
  }
  cudaStream_t s = c->stream;
  if (cudaMemsetAsync(c->x, 0, 3 * np * sizeof(double), s) ||
      cudaMemsetAsync(c->v, 0, 3 * np * sizeof(double), s) ||
      cudaMemsetAsync(c->m, 0, np * sizeof(double), s) ||
      cudaMemsetAsync(c->xbar, 0, 3 * np * sizeof(double), s) ||
      cudaMemsetAsync(c->vbar, 0, 3 * np * sizeof(double), s) ||
      cudaMemsetAsync(c->st, 0, np * sizeof(float4), s) ||
      cudaMemsetAsync(c->vst, 0, 2 * np * sizeof(float4), s) ||
      cudaMemsetAsync(c->status, 0, sizeof(int), s) ||
      cudaMemsetAsync(c->pctr, 0, (np / 128) * sizeof(unsigned), s) || upload_params(c)) {
    free_all(c);
    delete c;
    return NBODY_ECUDA;
  }
  *out = c;
  return NBODY_OK;
}

void nbody_destroy(nbody_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->gs) cudaStreamSynchronize(c->gs);
  drop_graphs(c);
  if (c->gs) cudaStreamDestroy(c->gs);
  if (c->gev_in) cudaEventDestroy(c->gev_in);
  if (c->gev_out) cudaEventDestroy(c->gev_out);
  if (c->batch) nb::batch_destroy(c->batch);
  c->batch = nullptr;
  free_all(c);
  delete c;
}

int nbody_set_params(nbody_ctx* c, const nbody_params* p) {
  if (!c) return NBODY_EINVAL;
  if (c->batch) {
    if (!p) return NBODY_EINVAL;
    for (int s = 0; s < c->n_sims; ++s) {
      int rc = check_params(&p[s]);
      if (rc) return rc;
      if ((p[s].checkpoint_every > 0) != (p[0].checkpoint_every > 0) || p[s].tape_mode != 0)
        return NBODY_EINVAL;
    }
    return nb::batch_set_params(c->batch, p);
  }
  int rc = check_params(p);
  if (rc) return rc;
  c->p = *p;
  c->acc_valid = false;
  c->tape_steps = 0;
  c->last_seg_valid = false;
  return upload_params(c);
}

int nbody_set_state(nbody_ctx* c, const double* x, const double* v,
                    const double* m) {
  if (!c || !x || !v || !m) return NBODY_EINVAL;
  if (c->batch) return nb::batch_set_state(c->batch, x, v, m);
  int rc;
  if ((rc = copy_in3(c, c->x, x)) || (rc = copy_in3(c, c->v, v)) ||
      (rc = copy_in(c->m, m, (size_t)c->n, c->stream)))
    return rc;
  c->acc_valid = false;
  c->tape_steps = 0;
  c->last_seg_valid = false;
  rc = upload_params(c);  // resets the guide; synchronises (pageable inputs)
  if (rc) return rc;
  // equal masses select the pair kernels that leave the mass out of the sum
  double mm[2];
  CK(nb::launch_minmax(c->m, c->n, c->red, c->stream));
  CK(cudaMemcpyAsync(mm, c->red, sizeof(mm), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const bool eqm = mm[0] == mm[1] && mm[0] > 0.0;
  if (!c->shape_fixed[0]) c->fcfg = nb::choose_pair_cfg(c->npad, c->sm_count, false, eqm);
  if (!c->shape_fixed[1]) c->vcfg = nb::choose_pair_cfg(c->npad, c->sm_count, true, eqm);
  c->fcfg.eqm = c->vcfg.eqm = eqm;
  c->m_eq = eqm ? mm[0] : 1.0;
  // stage masses (and positions) once; the update kernel rewrites positions
  CK(nb::launch_stage(c->x, c->m, c->fixed_center, c->n, c->npad, c->st,
                      c->stream));
  CK(cudaMemsetAsync(c->vst, 0, 2 * (size_t)c->npad * sizeof(float4), c->stream));
  return NBODY_OK;
}

int nbody_get_state(nbody_ctx* c, double* x, double* v) {
  if (!c) return NBODY_EINVAL;
  if (c->batch) return nb::batch_get_state(c->batch, x, v);
  int rc;
  if (x && (rc = copy_out3(c, x, c->x))) return rc;
  if (v && (rc = copy_out3(c, v, c->v))) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return NBODY_OK;
}

int nbody_step(nbody_ctx* c, int64_t k) {
  if (!c || k < 0) return NBODY_EINVAL;
  if (k == 0) return NBODY_OK;
  if (c->batch) return nb::batch_integrate(c->batch, k);
  return run_forward(c, k, false);
}

int nbody_integrate(nbody_ctx* c, int64_t n_steps, double* x_out,
                    double* v_out) {
  if (!c || n_steps < 1) return NBODY_EINVAL;
  if (c->batch) {
    int rc = nb::batch_integrate(c->batch, n_steps);
    if (rc) return rc;
    if (x_out || v_out) return nb::batch_get_state(c->batch, x_out, v_out);
    return NBODY_OK;
  }
  int rc = run_forward(c, n_steps, c->p.checkpoint_every > 0);
  if (rc) return rc;
  if (x_out || v_out) return nbody_get_state(c, x_out, v_out);
  return NBODY_OK;
}

}  // extern "C"

namespace {

// The external potential's adjoint terms of the point a.xk (cotangents: the
// current v-bar) on the side stream aside, beside the point's pair VJP on
// stream s; the adjoint kernel then reads them (a.ea).  Without an external
// potential or side stream, or outside the sizes where this pays, the
// adjoint kernel computes them itself (the same arithmetic).
int fork_ext_adjoint(nbody_ctx* c, nb::AdjointArgs& a, cudaStream_t s) {
  a.ea = nullptr;
  if (!c->p.ext_flags || !c->aside || !c->ea || !ext_adjoint_beside(c)) return NBODY_OK;
  CK(cudaEventRecord(c->ev_afork, s));
  CK(cudaStreamWaitEvent(c->aside, c->ev_afork, 0));
  CK(nb::launch_ext_adjoint(c->dp, a.xk, c->vbar, c->n, c->npad, c->ea, c->aside));
  CK(cudaEventRecord(c->ev_ajoin, c->aside));
  a.ea = c->ea;
  return NBODY_OK;
}

int join_ext_adjoint(nbody_ctx* c, const nb::AdjointArgs& a, cudaStream_t s) {
  if (a.ea) CK(cudaStreamWaitEvent(s, c->ev_ajoin, 0));
  return NBODY_OK;
}

// The launches of one reverse sweep over the recorded tape (on stream s):
// cotangent scaling, segment recomputation, pair VJP and adjoint update at
// every point, and the reduction of the parameter-gradient sums into red.
int record_sweep(nbody_ctx* c, cudaStream_t s) {
  const size_t np = (size_t)c->npad;
  Tape T{c, 3 * np};
  const int64_t n = c->tape_steps, K = c->K, nseg = c->nseg;
  const bool last_valid = c->last_seg_valid;
  CK(cudaMemsetAsync(c->lsc, 0, nb::kLscDoubles * sizeof(double), s));
  CK(nb::launch_lam_absmax(c->vbar, c->n, c->npad, c->lsc, (int)(n & 1), s));
  CK(nb::launch_stage_vjp(T.cpx(nseg), c->m, c->vbar, center_at(c, n), c->n,
                          c->npad, c->vst, c->lsc, (int)(n & 1), s));
  nb::AdjointArgs a{};
  a.P = c->dp;
  a.n = c->n;
  a.npad = c->npad;
  a.xbar = c->xbar;
  a.vbar = c->vbar;
  a.gpart = c->part;
  a.S = c->vcfg.S;
  a.mscale = c->vcfg.eqm ? c->m_eq : 1.0;
  a.m = c->m;
  a.vst = c->vst;
  a.blk = c->blk;
  a.lsc = c->lsc;
  a.mpart = c->want_mbar ? c->mpart : nullptr;
  a.mbar = c->want_mbar ? c->mbar : nullptr;
  a.status = c->status;
  double* mp = c->want_mbar ? c->mpart : nullptr;
  // with the VJP's slices summed in its kernel the adjoint reads one slice
  const bool vfin = use_fin(c->vcfg, c->vfin_mode);
  double* vfin_p = vfin ? c->fin : nullptr;
  if (vfin) {
    a.gpart = c->fin;
    a.S = 1;
    if (a.mpart) a.mpart = c->fin + 3 * np;
  }
  // small systems: segment sg - 1 is recomputed on rs2 (second buffer,
  // second scratch) while the reverse sweep of segment sg runs on s; the
  // last segment uses the first buffer (where the forward run keeps it)
  const bool overlap = use_overlap(c) && nseg >= 2;
  auto seg_of = [&](int64_t sg) { return ((nseg - 1 - sg) & 1) ? c->seg2 : c->seg; };
  // the update restages positions only: masses and padding come from the
  // primary staging
  if (overlap)
    CK(cudaMemcpyAsync(c->st2, c->st, np * sizeof(float4), cudaMemcpyDeviceToDevice, s));
  for (int64_t sg = nseg - 1; sg >= 0; --sg) {
    const int64_t k0 = sg * K;
    const int64_t Ks = (k0 + K <= n) ? K : n - k0;
    if (!overlap) {
      if (!(sg == nseg - 1 && last_valid)) {
        const int rc = recompute_segment(c, sg, s, primary_scratch(c), nullptr);
        if (rc) return rc;
      }
    } else {
      T.seg = seg_of(sg);
      if (sg == nseg - 1) {
        if (!last_valid) {
          const int rc = recompute_segment(c, sg, s, primary_scratch(c), T.seg);
          if (rc) return rc;
        }
      } else {
        CK(cudaStreamWaitEvent(s, c->ev_rready, 0));  // segment sg recomputed
      }
      if (sg >= 1) {  // segment sg - 1, beside this segment's reverse sweep
        CK(cudaEventRecord(c->ev_rfork, s));
        CK(cudaStreamWaitEvent(c->rs2, c->ev_rfork, 0));
        const int rc = recompute_segment(c, sg - 1, c->rs2, second_scratch(c), seg_of(sg - 1));
        if (rc) return rc;
        CK(cudaEventRecord(c->ev_rready, c->rs2));
      }
    }
    for (int64_t j = Ks; j >= 1; --j) {
      const int64_t k = k0 + j;
      a.xk = (j == Ks) ? T.cpx(sg + 1) : T.sx(j);
      if (int r_ = fork_ext_adjoint(c, a, s)) return r_;
      CK(timed(c, NBODY_KCLASS_VJP, [&] {
        return nb::launch_pair_vjp_fin(c->vcfg, c->vst, c->npad, c->hp.eps2f, c->part, mp,
                                       vfin_p, c->pctr, s);
      }));
      if (int r_ = join_ext_adjoint(c, a, s)) return r_;
      a.ak = (j == Ks) ? T.cpa(sg + 1) : T.sa(j);
      a.ck = (k == n) ? 0.5 : 1.0;
      a.drift = 1;
      a.vh_prev = T.svh(j);
      a.x_prev = T.sx(j - 1);
      a.c_prev = center_at(c, k - 1);
      a.slot = (int)(k & 1);
      CK(cudaMemsetAsync(c->lsc + 2 + (1 - a.slot), 0, sizeof(double), s));
      CK(timed(c, NBODY_KCLASS_ADJOINT, [&] { return nb::launch_adjoint(a, s); }));
    }
  }
  // point 0: opening half kick of the first step
  a.xk = T.cpx(0);
  if (int r_ = fork_ext_adjoint(c, a, s)) return r_;
  CK(timed(c, NBODY_KCLASS_VJP, [&] {
    return nb::launch_pair_vjp_fin(c->vcfg, c->vst, c->npad, c->hp.eps2f, c->part, mp, vfin_p,
                                   c->pctr, s);
  }));
  if (int r_ = join_ext_adjoint(c, a, s)) return r_;
  a.ak = T.cpa(0);
  a.ck = 0.5;
  a.drift = 0;
  a.vh_prev = nullptr;
  a.x_prev = nullptr;
  a.c_prev = nullptr;
  a.slot = 0;
  CK(timed(c, NBODY_KCLASS_ADJOINT, [&] { return nb::launch_adjoint(a, s); }));
  CK(nb::launch_reduce_rows(c->blk, c->nblk, nb::kAdjCols, c->red, s));
  return NBODY_OK;
}

}  // namespace

extern "C" {

int nbody_vjp(nbody_ctx* c, const double* xbar, const double* vbar,
              double* x0bar, double* v0bar, double* mbar_or_null,
              double theta_bar[4]) {
  if (!c || !theta_bar || c->batch) return NBODY_EINVAL;
  if (c->tape_steps < 1) return NBODY_ESTATE;
  cudaStream_t s = c->stream;
  const size_t np = (size_t)c->npad;
  int rc;
  c->want_mbar = mbar_or_null != nullptr;
  if (c->want_mbar) {
    if (!c->mpart) {
      drop_graphs(c);
      if ((rc = dalloc(&c->mpart, (size_t)c->Smax * np)) || (rc = dalloc(&c->mbar, np)))
        return rc;
    }
    CK(cudaMemsetAsync(c->mbar, 0, np * sizeof(double), s));
  }
  CK(cudaMemsetAsync(c->xbar, 0, 3 * np * sizeof(double), s));
  CK(cudaMemsetAsync(c->vbar, 0, 3 * np * sizeof(double), s));
  if (xbar && (rc = copy_in3(c, c->xbar, xbar))) return rc;
  if (vbar && (rc = copy_in3(c, c->vbar, vbar))) return rc;
  CK(cudaMemsetAsync(c->blk, 0, (size_t)c->nblk * nb::kAdjCols * sizeof(double), s));
  c->have_grad = false;
  if (graph_eligible(c, c->tape_steps)) {
    const uint64_t key[12] = {2, (uint64_t)c->tape_steps, (uint64_t)c->K, (uint64_t)c->nseg,
                              (uint64_t)c->last_seg_valid, (uint64_t)c->p.center_mode,
                              cfg_word(c->fcfg), cfg_word(c->vcfg), bits(c->m_eq),
                              (uint64_t)c->want_mbar, (uint64_t)use_fin(c->fcfg, c->fin_mode),
                              (uint64_t)use_fin(c->vcfg, c->vfin_mode)};
    rc = run_graph(c, key, [&](cudaStream_t gs) { return record_sweep(c, gs); });
  } else {
    rc = record_sweep(c, s);
  }
  if (rc) return rc;
  c->last_seg_valid = false;  // the segment buffer now holds segment 0
  if (x0bar && (rc = copy_out3(c, x0bar, c->xbar))) return rc;
  if (v0bar && (rc = copy_out3(c, v0bar, c->vbar))) return rc;
  if (mbar_or_null)
    CK(cudaMemcpyAsync(mbar_or_null, c->mbar, (size_t)c->n * sizeof(double), cudaMemcpyDefault, s));
  double h[nb::kAdjCols];
  CK(cudaMemcpyAsync(h, c->red, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int q = 0; q < 4; ++q) theta_bar[q] = h[q];
  // potential parameters in the order (M_NFW, r_s, M_MN, a_MN, b_MN, M_b)
  c->pot_bar[0] = h[2];
  c->pot_bar[1] = h[4];
  c->pot_bar[2] = h[3];
  c->pot_bar[3] = h[5];
  c->pot_bar[4] = h[6];
  c->pot_bar[5] = h[7];
  c->have_grad = true;
  int st = 0;
  CK(cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (st & nb::kStatusNaN) return NBODY_ENAN;
  return NBODY_OK;
}

int nbody_potential_grad(nbody_ctx* c, double out[6]) {
  if (!c || !out || c->batch) return NBODY_EINVAL;
  if (!c->have_grad) return NBODY_ESTATE;
  for (int q = 0; q < 6; ++q) out[q] = c->pot_bar[q];
  return NBODY_OK;
}

int nbody_energy(nbody_ctx* c, double out[4]) {
  if (!c || !out || c->batch) return NBODY_EINVAL;
  cudaStream_t s = c->stream;
  const double* cen = (c->p.center_mode == NBODY_CENTER_GUIDE) ? c->guide
                                                               : c->fixed_center;
  CK(nb::launch_stage(c->x, c->m, cen, c->n, c->npad, c->st, s));
  CK(nb::launch_pair_accel(c->fcfg, c->st, c->npad, c->hp.eps2f, c->part,
                           c->pot, s));
  const int nb_ = nb::energy_blocks(c->n);
  CK(cudaMemsetAsync(c->blk, 0, (size_t)nb_ * 6 * sizeof(double), s));
  CK(nb::launch_energy(c->dp, c->x, c->v, c->m, c->n, c->pot, c->fcfg.S,
                       c->npad, c->blk, nb_, s));
  CK(nb::launch_reduce_rows(c->blk, nb_, 6, c->red, s));
  double h[6];
  CK(cudaMemcpyAsync(h, c->red, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  out[0] = h[0];
  out[1] = h[1];
  out[2] = h[2];
  out[3] = std::sqrt(h[3] * h[3] + h[4] * h[4] + h[5] * h[5]);
  return NBODY_OK;
}

int nbody_momentum(nbody_ctx* c, double out[3]) {
  if (!c || !out || c->batch) return NBODY_EINVAL;
  double e[4];
  int rc = nbody_energy(c, e);
  if (rc) return rc;
  double h[8];
  CK(cudaMemcpyAsync(h, c->red, 6 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  out[0] = h[3];
  out[1] = h[4];
  out[2] = h[5];
  return NBODY_OK;
}

int nbody_get_status(nbody_ctx* c) {
  if (!c) return NBODY_EINVAL;
  if (c->batch) return nb::batch_status(c->batch);
  int st = 0;
  CK(cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (st & nb::kStatusNaN) return NBODY_ENAN;
  if (st & nb::kStatusTimeout) return NBODY_ETIMEOUT;
  return NBODY_OK;
}

int nbody_create_batch(nbody_ctx** out, int n_sims, const int64_t* offsets,
                       const nbody_params* p, void* cuda_stream) {
  if (!out) return NBODY_EINVAL;
  *out = nullptr;
  if (n_sims < 1 || !offsets || !p || offsets[0] != 0) return NBODY_EINVAL;
  for (int s = 0; s < n_sims; ++s) {
    if (offsets[s + 1] <= offsets[s]) return NBODY_EINVAL;
    int rc = check_params(&p[s]);
    if (rc) return rc;
    if ((p[s].checkpoint_every > 0) != (p[0].checkpoint_every > 0) || p[s].tape_mode != 0)
      return NBODY_EINVAL;
  }
  int dev = 0, sms = 0;
  int rc = check_device(&dev, &sms);
  if (rc) return rc;
  nbody_ctx* c = new (std::nothrow) nbody_ctx();
  if (!c) return NBODY_ENOMEM;
  c->dev = dev;
  c->sm_count = sms;
  c->n = offsets[n_sims];
  c->n_sims = n_sims;
  c->stream = (cudaStream_t)cuda_stream;
  c->p = p[0];
  rc = nb::batch_create(&c->batch, n_sims, offsets, p, c->stream, sms);
  if (rc) {
    delete c;
    return rc;
  }
  *out = c;
  return NBODY_OK;
}

int nbody_vjp_batch(nbody_ctx* c, const double* xbar, const double* vbar, double* x0bar,
                    double* v0bar, double* theta_bar) {
  if (!c || !c->batch) return NBODY_EINVAL;
  return nb::batch_vjp(c->batch, xbar, vbar, x0bar, v0bar, theta_bar);
}

int nbody_autotune(nbody_ctx* c, int64_t probe_steps, int* best,
                   double ms[NBODY_NTUNE]) {
  if (!c || !c->batch) return NBODY_EINVAL;
  return nb::batch_autotune(c->batch, probe_steps, best, ms);
}

int nbody_set_tuning(nbody_ctx* c, int choice) {
  if (!c || !c->batch) return NBODY_EINVAL;
  return nb::batch_set_tuning(c->batch, choice);
}

int nbody_get_tuning(nbody_ctx* c) {
  if (!c || !c->batch) return NBODY_EINVAL;
  return nb::batch_tuning(c->batch);
}

int nbody_set_pair_shape(nbody_ctx* c, int vjp, int variant, int threads,
                         int per_thread, int chunks) {
  if (!c || c->batch || (variant != 0 && variant != 1) || chunks < 0 || chunks > c->Smax)
    return NBODY_EINVAL;
  if (!nb::pair_shape_supported(variant, threads, per_thread, vjp != 0)) return NBODY_EINVAL;
  nb::PairCfg& cfg = vjp ? c->vcfg : c->fcfg;
  nb::PairCfg t = cfg;
  t.variant = variant;
  t.nt = threads;
  t.r = per_thread;
  t.vjp_tile_pairs = nb::choose_pair_cfg(c->npad, c->sm_count, vjp != 0, t.eqm).vjp_tile_pairs;
  if (t.variant == nb::kTile && c->npad % (t.nt * t.r) != 0) return NBODY_EINVAL;
  if (chunks == 0) {
    const int occ = vjp ? nb::vjp_blocks_per_sm(t) : nb::pair_blocks_per_sm(t);
    t.S = nb::choose_chunks(t, c->npad, c->sm_count, occ);
  } else {
    t.S = chunks;
  }
  cfg = t;
  drop_graphs(c);
  c->shape_fixed[vjp ? 1 : 0] = true;
  c->acc_valid = false;
  c->tape_steps = 0;
  c->last_seg_valid = false;
  return NBODY_OK;
}

int nbody_set_pair_tile(nbody_ctx* c, int vjp, int tile_pairs) {
  if (!c || c->batch) return NBODY_EINVAL;
  nb::PairCfg& cfg = vjp ? c->vcfg : c->fcfg;
  if (cfg.variant != nb::kTile) return NBODY_EINVAL;
  const int dflt = nb::choose_pair_cfg(c->npad, c->sm_count, vjp != 0, cfg.eqm).vjp_tile_pairs;
  if (tile_pairs != dflt && tile_pairs != 128) return NBODY_EINVAL;
  if (!nb::pair_tile_supported(cfg.nt, cfg.r, tile_pairs, vjp != 0)) return NBODY_EINVAL;
  if (c->npad % (2 * tile_pairs) != 0) return NBODY_EINVAL;
  cfg.vjp_tile_pairs = tile_pairs;
  drop_graphs(c);
  c->shape_fixed[vjp ? 1 : 0] = true;
  c->acc_valid = false;
  c->tape_steps = 0;
  c->last_seg_valid = false;
  return NBODY_OK;
}

int nbody_get_pair_tile(nbody_ctx* c, int vjp) {
  if (!c || c->batch) return NBODY_EINVAL;
  return (vjp ? c->vcfg : c->fcfg).vjp_tile_pairs;
}

int nbody_set_pair_finish(nbody_ctx* c, int vjp, int mode) {
  if (!c || c->batch || mode < -1 || mode > 1) return NBODY_EINVAL;
  (vjp ? c->vfin_mode : c->fin_mode) = mode;
  return NBODY_OK;
}

int nbody_get_pair_shape(nbody_ctx* c, int vjp, int out[4]) {
  if (!c || c->batch || !out) return NBODY_EINVAL;
  const nb::PairCfg& cfg = vjp ? c->vcfg : c->fcfg;
  out[0] = cfg.variant;
  out[1] = cfg.nt;
  out[2] = cfg.r;
  out[3] = cfg.S;
  return NBODY_OK;
}

int nbody_autotune_pair(nbody_ctx* c, int probe_launches, int fwd_best[4],
                        int vjp_best[4]) {
  if (!c || c->batch || probe_launches < 1) return NBODY_EINVAL;
  cudaStream_t s = c->stream;
  const bool eqm = c->fcfg.eqm;
  // stage the current positions (and zero cotangents) for both kernels
  const double* cen = (c->p.center_mode == NBODY_CENTER_GUIDE) ? c->guide : c->fixed_center;
  CK(nb::launch_stage(c->x, c->m, cen, c->n, c->npad, c->st, s));
  CK(cudaMemsetAsync(c->vbar, 0, 3 * (size_t)c->npad * sizeof(double), s));
  CK(cudaMemsetAsync(c->lsc, 0, nb::kLscDoubles * sizeof(double), s));
  CK(nb::launch_stage_vjp(c->x, c->m, c->vbar, cen, c->n, c->npad, c->vst, c->lsc, 0, s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  struct Shape {
    int variant, nt, r, tj;  // tj = 0: the kernel's default tile
  };
  const Shape fwd[] = {{0, 128, 4, 0},   {0, 128, 8, 0},   {0, 256, 4, 0}, {0, 256, 2, 0},
                       {0, 128, 2, 0},   {0, 128, 1, 0},   {1, 256, 4, 0}, {1, 256, 8, 0},
                       {0, 128, 4, 128}, {0, 128, 2, 128}, {0, 128, 1, 128},
                       {0, 64, 2, 128},  {0, 64, 4, 128},  {0, 64, 2, 0}};
  const Shape vjp[] = {{0, 256, 2, 0}, {0, 128, 4, 0}, {0, 128, 2, 0}, {0, 128, 1, 0},
                       {1, 256, 4, 0}, {1, 256, 2, 0}, {0, 64, 2, 0},
                       {0, 128, 2, 128}, {0, 128, 1, 128}, {0, 64, 2, 128}};
  int rc = NBODY_OK;
  int best_fin[2] = {0, 0};
  for (int which = 0; which < 2 && rc == NBODY_OK; ++which) {
    const Shape* list = which ? vjp : fwd;
    const int cnt = which ? (int)(sizeof(vjp) / sizeof(vjp[0])) : (int)(sizeof(fwd) / sizeof(fwd[0]));
    nb::PairCfg best = which ? c->vcfg : c->fcfg;
    double best_ms = 1e300;
    for (int k = 0; k < cnt && rc == NBODY_OK; ++k) {
      nb::PairCfg t = best;
      t.variant = list[k].variant;
      t.nt = list[k].nt;
      t.r = list[k].r;
      t.eqm = eqm;
      t.vjp_tile_pairs = list[k].tj ? list[k].tj
                                    : nb::choose_pair_cfg(c->npad, c->sm_count, which == 1, eqm)
                                          .vjp_tile_pairs;
      if (t.variant == nb::kTile && c->npad % (2 * t.vjp_tile_pairs) != 0) continue;
      if (t.variant == nb::kTile && (c->npad < 2048 || c->npad % (t.nt * t.r) != 0)) continue;
      if (t.variant == nb::kWarp && c->npad % (8 * t.r) != 0) continue;
      const int occ = which ? nb::vjp_blocks_per_sm(t) : nb::pair_blocks_per_sm(t);
      const int S0 = nb::choose_chunks(t, c->npad, c->sm_count, occ);
      // besides the occupancy-based chunk count, the nearest counts that
      // split the j-tiles evenly (equal work per block)
      int cand[3] = {S0, 0, 0};
      if (t.variant == nb::kTile) {
        const int64_t ntiles = c->npad / (2 * t.vjp_tile_pairs);
        for (int d = S0; d >= 1; --d)
          if (ntiles % d == 0) { cand[1] = d; break; }
        for (int d = S0 + 1; d <= std::min<int64_t>(ntiles, c->Smax); ++d)
          if (ntiles % d == 0) { cand[2] = d; break; }
      }
      // every candidate is timed with a consumer of its sums, the update
      // (kick 0, no drift: the state is left as it is; for the VJP it stands
      // in for the adjoint, which reads the same slices), once with the
      // slices summed by the consumer and once in the pair kernel
      for (int ci = 0; ci < 6 && rc == NBODY_OK; ++ci) {
        const int cs = ci % 3, fin = ci / 3;
        if (cand[cs] < 1 || cand[cs] > c->Smax || (cs > 0 && (cand[cs] == S0 ||
                                                           (cs == 2 && cand[2] == cand[1]))))
          continue;
        if (fin && (t.variant != nb::kTile || cand[cs] < 2)) continue;
        t.S = cand[cs];
        nb::UpdateArgs u = base_update(c, c->x, c->v);
        u.S = fin ? 1 : t.S;
        u.part = fin ? c->fin : c->part;
        u.mscale = 0.0;
        auto launch = [&]() {
          double* f = fin ? c->fin : nullptr;
          const cudaError_t e =
              which ? nb::launch_pair_vjp_fin(t, c->vst, c->npad, c->hp.eps2f, c->part, nullptr,
                                              f, c->pctr, s)
                    : nb::launch_pair_accel_fin(t, c->st, c->npad, c->hp.eps2f, c->part, f,
                                                c->pctr, s);
          return e == cudaSuccess ? nb::launch_update(u, s) : e;
        };
        if (launch() != cudaSuccess) {
          rc = NBODY_ECUDA;
          break;
        }
        // one timed launch sets the repetition count: at least probe_launches
        // and about 2 ms of launches, so that short kernels are timed well
        float ms1 = 0.f;
        if (cudaEventRecord(e0, s) != cudaSuccess || launch() != cudaSuccess ||
            cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
          rc = NBODY_ECUDA;
          break;
        }
        cudaEventElapsedTime(&ms1, e0, e1);
        int reps = probe_launches;
        if (ms1 > 0.f && 2.0f / ms1 > (float)reps) reps = (int)std::min(2.0f / ms1, 400.0f);
        if (cudaEventRecord(e0, s) != cudaSuccess) rc = NBODY_ECUDA;
        for (int q = 0; q < reps && rc == NBODY_OK; ++q)
          if (launch() != cudaSuccess) rc = NBODY_ECUDA;
        if (rc || cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
          rc = NBODY_ECUDA;
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)reps;
        if (ms < best_ms) {
          best_ms = ms;
          best = t;
          best_fin[which] = fin;
        }
      }
    }
    if (which) {
      c->vcfg = best;
      c->vfin_mode = best_fin[1];
      if (vjp_best) {
        vjp_best[0] = best.variant; vjp_best[1] = best.nt; vjp_best[2] = best.r; vjp_best[3] = best.S;
      }
    } else {
      c->fcfg = best;
      c->fin_mode = best_fin[0];
      if (fwd_best) {
        fwd_best[0] = best.variant; fwd_best[1] = best.nt; fwd_best[2] = best.r; fwd_best[3] = best.S;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->shape_fixed[0] = c->shape_fixed[1] = true;
  c->acc_valid = false;
  c->tape_steps = 0;
  c->last_seg_valid = false;
  return rc;
}

int nbody_set_timing(nbody_ctx* c, int enable) {
  if (!c || c->batch) return NBODY_EINVAL;
  c->timing = enable != 0;
  for (auto& u : c->ev_used) u = 0;
  return NBODY_OK;
}

int nbody_kernel_times(nbody_ctx* c, double ms[NBODY_NKCLASS],
                       int64_t launches[NBODY_NKCLASS]) {
  if (!c || !ms || c->batch) return NBODY_EINVAL;
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < NBODY_NKCLASS; ++k) {
    double t = 0.0;
    for (size_t i = 0; i < c->ev_used[k]; ++i) {
      float e = 0.f;
      CK(cudaEventElapsedTime(&e, c->ev[k][i].first, c->ev[k][i].second));
      t += e;
    }
    ms[k] = t;
    if (launches) launches[k] = (int64_t)c->ev_used[k];
    c->ev_used[k] = 0;
  }
  return NBODY_OK;
}

int nbody_pair_accel(int64_t n, const double* x, const double* m, double G,
                     double eps, const double center[3], double* acc,
                     void* cuda_stream) {
  if (n < 1 || !x || !m || !acc || !center || !(eps > 0.0)) return NBODY_EINVAL;
  int dev = 0, sms = 0;
  int rc = check_device(&dev, &sms);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int64_t npad = ((n + nb::kPad - 1) / nb::kPad) * nb::kPad;
  const nb::PairCfg cfg = nb::choose_pair_cfg(npad, sms, false, false);
  // scratch: padded SoA copy of x and m, centre, staging, partials
  const size_t bytes_x = (size_t)4 * npad * sizeof(double);
  const size_t bytes_st = (size_t)npad * sizeof(float4);
  const size_t bytes_part = (size_t)cfg.S * 3 * npad * sizeof(double);
  char* buf = nullptr;
  if (cudaMallocAsync((void**)&buf, bytes_x + 256 + bytes_st + bytes_part, s) !=
      cudaSuccess) {
    cudaGetLastError();
    return NBODY_ENOMEM;
  }
  double* xp = (double*)buf;
  double* mp = xp + 3 * npad;
  double* cen = (double*)(buf + bytes_x);
  float4* st = (float4*)(buf + bytes_x + 256);
  double* part = (double*)(buf + bytes_x + 256 + bytes_st);
  rc = NBODY_OK;
  cudaError_t e = cudaMemsetAsync(xp, 0, bytes_x, s);
  for (int d = 0; d < 3 && e == cudaSuccess; ++d)
    e = cudaMemcpyAsync(xp + (size_t)d * npad, x + (size_t)d * n,
                        (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(mp, m, (size_t)n * sizeof(double),
                        cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cen, center, 3 * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = nb::launch_stage(xp, mp, cen, n, npad, st, s);
  if (e == cudaSuccess)
    e = nb::launch_pair_accel(cfg, st, npad, (float)(eps * eps), part, nullptr, s);
  if (e == cudaSuccess) e = nb::launch_reduce_partials(part, cfg.S, npad, n, G, acc, s);
  if (e != cudaSuccess) rc = NBODY_ECUDA;
  // the centre copy reads host memory: finish it before returning
  if (cudaStreamSynchronize(s) != cudaSuccess) rc = NBODY_ECUDA;
  cudaFreeAsync(buf, s);
  return rc;
}

int nbody_ext_accel(const nbody_params* p, int64_t n, const double* x, double* acc,
                    void* cuda_stream) {
  if (!p || n < 1 || !x || !acc) return NBODY_EINVAL;
  int rc = check_params(p);
  if (rc) return rc;
  int dev = 0, sms = 0;
  if ((rc = check_device(&dev, &sms))) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t bytes = (size_t)3 * n * sizeof(double);
  double* buf = nullptr;
  if (cudaMallocAsync((void**)&buf, 2 * bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return NBODY_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(buf, x, bytes, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = nb::launch_ext_accel(to_dev(*p), buf, n, buf + 3 * n, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(acc, buf + 3 * n, bytes, cudaMemcpyDefault, s);
  rc = e == cudaSuccess ? NBODY_OK : NBODY_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) rc = NBODY_ECUDA;
  cudaFreeAsync(buf, s);
  return rc;
}

}  // extern "C"
