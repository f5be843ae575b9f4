// gd_host.cu -- C ABI, multigrid planning and the solve driver (host code).
//
// Structure of one solve (gd_diffuse_z / gd_screened_poisson_slices):
//   x  <- x0 (default: 0 for AD, I0 for SP), held as a float pair (hi, lo)
//   r  <- b - A x                    (outer pass, float-pair differences)
//   repeat: e <- V(nu1,nu2)-cycle on A e = r from e = 0   (FP32 hierarchy)
//           x <- x + e (+ mean shift for AD);  r <- b - A x;  ||r|| read back
//   until ||r|| <= rel_tol ||b||.
// The V-cycle itself is the paper's (Sec. 4.1): relax, compute the residual
// and down-sample it to the next level's constraints, ..., direct solve at
// the coarsest level, up-sample and add the correction, relax again.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <memory>
#include <vector>

#include "gd.h"
#include "gd_internal.h"

namespace {

enum ProfClass {
  P_SWEEP_FINE = 0,
  P_SWEEP_COARSE,
  P_RESTRICT,
  P_PROLONG,
  P_OUTER,
  P_COARSEST,
  P_REDUCE,
  P_COPY,
  P_NUM
};
const char *kProfNames[P_NUM] = {"rb_sweep_fine", "rb_sweep_coarse", "residual_restrict",
                                 "prolong_add",   "outer_update_residual", "coarsest_fdm",
                                 "reduce",        "copy"};

struct Level {
  LevelDev d;
  int fx = 0, fy = 0, fz = 0;  // axes coarsened from this level to the next
  // the level's arrays: float32, or bfloat16 (esz = 2) in the mixed mode, where
  // the buffers hold n halves
  float *x = nullptr, *b = nullptr, *t = nullptr;
  size_t n = 0;
  int esz = 4;
  // Hybrid discretisation: the level's per-axis Galerkin factors
  float *hf = nullptr;
  HLevelDev hd{};
};

// internal system id of the general screened Poisson solve (explicit b)
constexpr int SYS_GENERIC = 2;

struct ProfRec {
  int cls;
  cudaEvent_t a, b;
  double bytes;
};

// A V-cycle captured as a CUDA graph.  Every cycle of a solve launches the
// same kernels on the same buffers (each level's ping-pong pointers return to
// their start after an even number of sweeps), so one capture serves all of
// them.  With profiling on, the per-kernel event pairs are graph nodes too.
struct VGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<ProfRec> recs;
  long long launches = 0;  // kernels per replay
  int nu1 = 0, nu2 = 0;
  bool zero_init = false, sum_e = false, prof = false, usable = false;
};

// A multigrid hierarchy for one set of weights.  Level 0's three arrays are
// the stack's fine workspace, shared by all cached plans (one solve runs at a
// time); coarser levels, the coarsest-level factors and the captured
// V-cycle graphs belong to the plan.
struct Plan {
  bool valid = false;
  int batch_z = 0;
  double w[4] = {0, 0, 0, 0};  // alpha, bx, by, bz
  int cxy = 16;
  int prec = GD_PREC_FP32;     // requested storage (the cache key)
  bool half = false;           // levels above the coarsest hold bfloat16
  std::vector<Level> L;
  float *Vx = nullptr, *Vy = nullptr, *Vz = nullptr, *Dinv = nullptr;
  // Linear: the fine factors scaled to integers (mass factors times lscale)
  float *lfac = nullptr;
  HLevelDev ls{};
  double lscale[3] = {1.0, 1.0, 1.0};
  std::vector<std::unique_ptr<VGraph>> graphs;
  unsigned long long last_use = 0;
};

// Plans kept per stack: a solve alternating AD and SP (or a few weight sets)
// rebuilds nothing after the first use of each.
constexpr int kMaxPlans = 4;

}  // namespace

struct gd_stack {
  int nx = 0, ny = 0, nz = 0, bc = 0, disc = 0, prec = 0;
  int device = -1;  // the device current at creation (-1: none): caller device arrays must live there
  cudaStream_t stream = nullptr;
  std::vector<std::unique_ptr<Plan>> plans;  // cache, least recently used evicted
  Plan *cur = nullptr;                       // the plan of the running call
  unsigned long long use_clock = 0;
  float *f_x = nullptr, *f_b = nullptr, *f_t = nullptr;  // fine-level workspace
  // fine-level outer iterate buffers (second float pair, low parts)
  float *xh2 = nullptr, *xl1 = nullptr, *xl2 = nullptr;
  float *lbh = nullptr;  // Linear discretisation: high part of the right-hand side
  float *i1 = nullptr;   // gd_ad_then_sp: the intermediate I1 on the device
  double *partials = nullptr;
  int partials_cap = 0;  // blocks
  double *scalars = nullptr;
  double *h_scalars = nullptr;  // pinned
  // staging buffers for host pointers
  float *stage[4] = {nullptr, nullptr, nullptr, nullptr};
  // profiling
  bool prof_on = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> ev_pool;
  long long prof_launches[P_NUM] = {0};
  double prof_ms[P_NUM] = {0}, prof_bytes[P_NUM] = {0};
  long long launches = 0;
  bool no_tma = false;     // GD_DISABLE_TMA set at creation: plain (unfused) kernels only
  bool no_graph = false;   // GD_DISABLE_GRAPHS set at creation: direct launches only
  long long fail_alloc_after = -1;  // GD_FAIL_ALLOC_AFTER at creation: fault injection on the host
  long long allocs = 0;
  std::vector<VGraph *> replayed;  // graphs replayed since the last collection (profiling)
  cudaStream_t cap_stream = nullptr;
  bool capturing = false;  // events become graph nodes (external event records)
  std::string err;
};

namespace {

void set_err(gd_stack *s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (s) s->err = buf;
}

#define CK(call)                                                                    \
  do {                                                                              \
    cudaError_t _e = (call);                                                        \
    if (_e != cudaSuccess) {                                                        \
      set_err(s, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e), __FILE__, \
              __LINE__);                                                            \
      return GD_ERR_CUDA;                                                           \
    }                                                                               \
  } while (0)

int report(gd_report *rep, int st) {
  if (rep) rep->status = st;
  return st;
}

// ---- profiling ----
cudaEvent_t ev_get(gd_stack *s) {
  if (!s->ev_pool.empty()) {
    cudaEvent_t e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

struct ProfScope {
  gd_stack *s;
  int cls;
  double bytes;
  cudaEvent_t a = nullptr;
  ProfScope(gd_stack *s_, int cls_, double bytes_) : s(s_), cls(cls_), bytes(bytes_) {
    ++s->launches;
    if (s->prof_on && s->recs.size() < 200000) {
      a = ev_get(s);
      record(a);
    }
  }
  void record(cudaEvent_t e) {
    if (s->capturing)
      cudaEventRecordWithFlags(e, s->stream, cudaEventRecordExternal);
    else
      cudaEventRecord(e, s->stream);
  }
  ~ProfScope() {
    if (a && bytes <= 0.0) {
      // cancelled: nothing was launched.  A captured record is a graph node
      // now, so the event stays with the graph (class -1 is never summed).
      if (s->capturing)
        s->recs.push_back(ProfRec{-1, a, nullptr, 0.0});
      else
        s->ev_pool.push_back(a);
      a = nullptr;
    }
    if (a) {
      cudaEvent_t b = ev_get(s);
      record(b);
      s->recs.push_back(ProfRec{cls, a, b, bytes});
    }
  }
};

void prof_collect(gd_stack *s) {
  if (s->recs.empty()) return;
  cudaStreamSynchronize(s->stream);
  for (auto &r : s->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      s->prof_ms[r.cls] += ms;
      s->prof_launches[r.cls] += 1;
      s->prof_bytes[r.cls] += r.bytes;
    }
    s->ev_pool.push_back(r.a);
    s->ev_pool.push_back(r.b);
  }
  s->recs.clear();
}

// Adds the timings of graphs replayed since the last call (their event pairs
// hold the latest replay); the stream must have been synchronised.
void prof_collect_graphs(gd_stack *s) {
  for (VGraph *g : s->replayed) {
    for (auto &r : g->recs) {
      if (r.cls < 0) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
        s->prof_ms[r.cls] += ms;
        s->prof_launches[r.cls] += 1;
        s->prof_bytes[r.cls] += r.bytes;
      }
    }
  }
  s->replayed.clear();
}

void release_recs(gd_stack *s, std::vector<ProfRec> &recs) {
  for (auto &r : recs) {
    if (r.a) s->ev_pool.push_back(r.a);
    if (r.b) s->ev_pool.push_back(r.b);
  }
  recs.clear();
}

void graphs_free(gd_stack *s, Plan &P) {
  for (auto &g : P.graphs) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    release_recs(s, g->recs);
  }
  P.graphs.clear();
}

// ---- device memory helpers ----
int dalloc(gd_stack *s, float **p, size_t n) {
  if (n == 0) n = 1;
  if (s->fail_alloc_after >= 0 && s->allocs >= s->fail_alloc_after) {
    // injected failure (host side): the allocation is refused as if the
    // device were out of memory
    *p = nullptr;
    set_err(s, "allocation %lld refused by GD_FAIL_ALLOC_AFTER=%lld (injected)", s->allocs,
            s->fail_alloc_after);
    return GD_ERR_OOM;
  }
  ++s->allocs;
  cudaError_t e = cudaMalloc((void **)p, n * sizeof(float));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    set_err(s, "cudaMalloc of %zu floats failed: %s", n, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? GD_ERR_OOM : GD_ERR_CUDA;
  }
  return GD_OK;
}

void dfree(float *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

// Frees what the plan owns (level 0's arrays are the stack's); the stream
// must be idle and the plan's graph timings collected.
void plan_free(gd_stack *s, Plan &P) {
  graphs_free(s, P);
  for (size_t li = 1; li < P.L.size(); ++li) {
    dfree(P.L[li].x);
    dfree(P.L[li].b);
    dfree(P.L[li].t);
  }
  for (auto &l : P.L) dfree(l.hf);
  dfree(P.lfac);
  P.L.clear();
  dfree(P.Vx);
  dfree(P.Vy);
  dfree(P.Vz);
  dfree(P.Dinv);
  P.valid = false;
}

int ensure_partials(gd_stack *s, int blocks) {
  if (blocks <= s->partials_cap) return GD_OK;
  if (s->partials) cudaFree(s->partials);
  s->partials = nullptr;
  s->partials_cap = 0;
  size_t cap = (size_t)blocks + 1024;
  if (cudaMalloc((void **)&s->partials, cap * S_NUM * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    set_err(s, "cudaMalloc of the partial-sum buffer failed");
    return GD_ERR_OOM;
  }
  s->partials_cap = (int)cap;
  return GD_OK;
}

// Build the multigrid hierarchy for weights w = (alpha, bx, by, bz).
// Coarsening (anisotropy-aware semi-coarsening): the interior coupling of
// axis d at a level is c_d = w_d * s_e * s_f (the other axes' children
// counts); an axis is halved (n_c = ceil(n/2)) when c_d >= max_d' c_d' / 2
// and it may still be coarsened (x, y: n >= 2*cxy; z: n >= 2 and coupled).
// When the strongest axis can no longer be halved the level is the coarsest.
// Coarse stiffness w_d is halved per coarsening of axis d (6-point stencil
// re-discretised at the coarse spacing); masses are the children counts.
int plan_build_into(gd_stack *s, Plan &P, const double w[4], int batch_z, int cxy, int prec);

// Makes the plan for these weights current: from the cache, else built (the
// least recently used plan is freed when the cache is full).
int plan_build(gd_stack *s, const double w[4], int batch_z, int cxy, int prec = GD_PREC_FP32) {
  s->cur = nullptr;
  for (auto &p : s->plans)
    if (p->valid && p->batch_z == batch_z && p->cxy == cxy && p->prec == prec &&
        std::memcmp(p->w, w, sizeof(p->w)) == 0) {
      p->last_use = ++s->use_clock;
      s->cur = p.get();
      return GD_OK;
    }
  CK(cudaStreamSynchronize(s->stream));
  if (!s->replayed.empty()) prof_collect_graphs(s);
  if ((int)s->plans.size() >= kMaxPlans) {
    size_t v = 0;
    for (size_t k = 1; k < s->plans.size(); ++k)
      if (s->plans[k]->last_use < s->plans[v]->last_use) v = k;
    plan_free(s, *s->plans[v]);
    s->plans.erase(s->plans.begin() + v);
  }
  const size_t n = (size_t)s->nx * s->ny * s->nz;
  int st;
  if (!s->f_x && (st = dalloc(s, &s->f_x, n)) != GD_OK) return st;
  if (!s->f_b && (st = dalloc(s, &s->f_b, n)) != GD_OK) return st;
  if (!s->f_t && (st = dalloc(s, &s->f_t, n)) != GD_OK) return st;
  std::unique_ptr<Plan> P(new Plan);
  if ((st = plan_build_into(s, *P, w, batch_z, cxy, prec)) != GD_OK) {
    plan_free(s, *P);
    return st;
  }
  P->last_use = ++s->use_clock;
  s->cur = P.get();
  s->plans.push_back(std::move(P));
  return GD_OK;
}

int plan_build_into(gd_stack *s, Plan &P, const double w[4], int batch_z, int cxy, int prec) {
  P.batch_z = batch_z;
  P.prec = prec;
  P.cxy = cxy;
  std::memcpy(P.w, w, sizeof(P.w));
  Level l0;
  l0.d = LevelDev{s->nx, s->ny, s->nz, 1, 1, 1, 1, 1, 1, (float)w[1], (float)w[2],
                  batch_z ? 0.f : (float)w[3], (float)w[0]};
  P.L.push_back(l0);
  double wd[3] = {w[1], w[2], batch_z ? 0.0 : w[3]};
  for (int guard = 0; guard < 64; ++guard) {
    Level &F = P.L.back();
    const LevelDev &d = F.d;
    const bool can[3] = {d.nx >= 2 * cxy, d.ny >= 2 * cxy, d.nz >= 2 && wd[2] > 0.0};
    const double c[3] = {wd[0] * d.sy * d.sz, wd[1] * d.sx * d.sz, wd[2] * d.sx * d.sy};
    const double cm = std::fmax(c[0], std::fmax(c[1], c[2]));
    int f[3];
    for (int a = 0; a < 3; ++a) f[a] = can[a] && c[a] > 0.0 && c[a] >= 0.5 * cm;
    if (!f[0] && !f[1] && !f[2]) break;
    F.fx = f[0];
    F.fy = f[1];
    F.fz = f[2];
    Level C;
    const int n[3] = {d.nx, d.ny, d.nz}, sf[3] = {d.sx, d.sy, d.sz}, lf[3] = {d.lx, d.ly, d.lz};
    int nn[3], ns[3], nl[3];
    for (int a = 0; a < 3; ++a) {
      if (f[a]) {
        nn[a] = (n[a] + 1) / 2;
        ns[a] = 2 * sf[a];
        nl[a] = (n[a] % 2 == 0) ? sf[a] + lf[a] : lf[a];
        wd[a] *= 0.5;
      } else {
        nn[a] = n[a];
        ns[a] = sf[a];
        nl[a] = lf[a];
      }
    }
    C.d = LevelDev{nn[0], nn[1], nn[2], ns[0], ns[1], ns[2], nl[0], nl[1], nl[2],
                   (float)wd[0], (float)wd[1], (float)wd[2], (float)w[0]};
    P.L.push_back(C);
  }
  // Mixed precision (the paper's 16-bit storage of intermediate solutions
  // and constraints, Sec. 4.1 "Disk I/O"): every level between the fine and
  // the coarsest stores its correction, constraints and sweep array as
  // bfloat16, when all of them meet TMA's row alignment (nx % 8); arithmetic
  // stays float32, and the fine level and the coarsest solve stay float32
  // (bfloat16 rounding of the fine correction is high-frequency noise that A
  // amplifies by its largest eigenvalue, which costs an AD cycle).
  P.half = prec == GD_PREC_MIXED && !s->no_tma && P.L.size() > 2 && zmarch_usable(P.L[0].d, 4);
  for (size_t li = 1; li + 1 < P.L.size() && P.half; ++li)
    P.half = zmarch_usable(P.L[li].d, 2);
  // workspace
  for (size_t li = 0; li < P.L.size(); ++li) {
    Level &l = P.L[li];
    l.n = (size_t)l.d.nx * l.d.ny * l.d.nz;
    l.esz = (P.half && li > 0 && li + 1 < P.L.size()) ? 2 : 4;
    if (li == 0) {
      l.x = s->f_x;
      l.b = s->f_b;
      l.t = s->f_t;
      continue;
    }
    int st;
    const size_t nf = l.esz == 2 ? (l.n + 1) / 2 : l.n;  // floats holding the level's values
    if ((st = dalloc(s, &l.x, nf)) != GD_OK) return st;
    if ((st = dalloc(s, &l.b, nf)) != GD_OK) return st;
    if ((st = dalloc(s, &l.t, nf)) != GD_OK) return st;
  }
  // Hybrid: per-axis Galerkin factors (K_d, M_d) of every level, from the
  // fine (1D Neumann Laplacian, identity) through P^T . P along halved axes
  // Linear: the fine mass factors are the P1 mass (1/6) tridiag(1, [2, 4,
  // ..., 4, 2], 1) (an axis of one node, or the z axis of independent
  // slices, keeps M = I)
  const bool hybrid = s->disc != GD_DISC_CONSTANT;
  const bool p1 = s->disc == GD_DISC_LINEAR;
  std::vector<double> HK[3], HM[3];
  if (hybrid) {
    const int n0[3] = {s->nx, s->ny, s->nz};
    for (int a = 0; a < 3; ++a) {
      const int n = n0[a];
      HK[a].assign((size_t)n * 3, 0.0);
      HM[a].assign((size_t)n * 3, 0.0);
      for (int i = 0; i < n; ++i) {
        if (i > 0) {
          HK[a][(size_t)i * 3 + 0] = -1.0;
          HK[a][(size_t)i * 3 + 1] += 1.0;
        }
        if (i < n - 1) {
          HK[a][(size_t)i * 3 + 2] = -1.0;
          HK[a][(size_t)i * 3 + 1] += 1.0;
        }
        HM[a][(size_t)i * 3 + 1] = 1.0;
      }
      if (p1 && n > 1 && !(a == 2 && batch_z))
        for (int i = 0; i < n; ++i) {
          HM[a][(size_t)i * 3 + 0] = i > 0 ? 1.0 / 6.0 : 0.0;
          HM[a][(size_t)i * 3 + 2] = i < n - 1 ? 1.0 / 6.0 : 0.0;
          HM[a][(size_t)i * 3 + 1] = (i > 0 ? 2.0 / 6.0 : 0.0) + (i < n - 1 ? 2.0 / 6.0 : 0.0);
        }
    }
    for (size_t li = 0; li < P.L.size(); ++li) {
      Level &l = P.L[li];
      if (li > 0) {
        const Level &f = P.L[li - 1];
        const int fl[3] = {f.fx, f.fy, f.fz}, nf[3] = {f.d.nx, f.d.ny, f.d.nz};
        for (int a = 0; a < 3; ++a)
          if (fl[a]) {
            std::vector<double> t;
            galerkin_tri(nf[a], HK[a], t);
            HK[a].swap(t);
            galerkin_tri(nf[a], HM[a], t);
            HM[a].swap(t);
          }
      }
      const int nn[3] = {l.d.nx, l.d.ny, l.d.nz};
      std::vector<float> h;
      for (int a = 0; a < 3; ++a) {
        for (int q = 0; q < 3 * nn[a]; ++q) h.push_back((float)HK[a][q]);
        for (int q = 0; q < 3 * nn[a]; ++q) h.push_back((float)HM[a][q]);
      }
      int st;
      if ((st = dalloc(s, &l.hf, h.size())) != GD_OK) return st;
      CK(cudaMemcpyAsync(l.hf, h.data(), h.size() * 4, cudaMemcpyHostToDevice, s->stream));
      CK(cudaStreamSynchronize(s->stream));
      const float *b0 = l.hf;
      l.hd = HLevelDev{l.d.nx, l.d.ny, l.d.nz, (float)w[1], (float)w[2], batch_z ? 0.f : (float)w[3],
                       (float)w[0], b0, b0 + 3 * nn[0], b0 + 6 * nn[0], b0 + 6 * nn[0] + 3 * nn[1],
                       b0 + 6 * nn[0] + 6 * nn[1], b0 + 6 * nn[0] + 6 * nn[1] + 3 * nn[2]};
      // uniform interior rows and their 27 coefficients (same float formula
      // as the kernels' general path)
      {
        const int fz = !batch_z && l.d.nz > 1 ? 1 : 0;
        for (int a = 0; a < 3; ++a) {
          const int n = nn[a], mid = n / 2;
          int lo = 1, hi = n - 2;
          auto same = [&](int r) {
            for (int d = 0; d < 3; ++d)
              if ((float)HK[a][(size_t)r * 3 + d] != (float)HK[a][(size_t)mid * 3 + d] ||
                  (float)HM[a][(size_t)r * 3 + d] != (float)HM[a][(size_t)mid * 3 + d])
                return false;
            return true;
          };
          if (n < 3) {
            lo = 1;
            hi = 0;
          } else {
            lo = mid;
            hi = mid;
            while (lo - 1 >= 1 && same(lo - 1)) --lo;
            while (hi + 1 <= n - 2 && same(hi + 1)) ++hi;
          }
          l.hd.ilo[a] = lo;
          l.hd.ihi[a] = hi;
        }
        if (!fz) {
          l.hd.ilo[2] = 0;
          l.hd.ihi[2] = l.d.nz - 1;
        }
        const int mx_ = nn[0] / 2, my_ = nn[1] / 2, mz_ = nn[2] / 2;
        for (int c = -1; c <= 1; ++c)
          for (int b = -1; b <= 1; ++b)
            for (int a = -1; a <= 1; ++a) {
              float v = 0.f;
              if (fz || c == 0) {
                const float mzc = (float)HM[2][(size_t)mz_ * 3 + c + 1];  // (the z diagonal when uncoupled)
                const float kzc = fz ? (float)HK[2][(size_t)mz_ * 3 + c + 1] : 0.f;
                const float zterm = l.hd.wz * kzc + l.hd.wm * mzc;
                const float myb = (float)HM[1][(size_t)my_ * 3 + b + 1], kyb = (float)HK[1][(size_t)my_ * 3 + b + 1];
                const float yz = myb * zterm + l.hd.wy * kyb * mzc;
                const float xz = l.hd.wx * myb * mzc;
                v = (float)HM[0][(size_t)mx_ * 3 + a + 1] * yz + (float)HK[0][(size_t)mx_ * 3 + a + 1] * xz;
              }
              l.hd.cst[(c + 1) * 9 + (b + 1) * 3 + (a + 1)] = v;
            }
      }
      if (li == 0 && p1) {
        // integer-scaled fine factors for the compensated outer pass
        std::vector<float> g;
        for (int a = 0; a < 3; ++a) {
          const bool mass_p1 = nn[a] > 1 && !(a == 2 && batch_z);
          P.lscale[a] = mass_p1 ? 6.0 : 1.0;
          for (int q = 0; q < 3 * nn[a]; ++q) g.push_back((float)HK[a][q]);
          for (int q = 0; q < 3 * nn[a]; ++q) g.push_back((float)std::nearbyint(HM[a][q] * P.lscale[a]));
        }
        if ((st = dalloc(s, &P.lfac, g.size())) != GD_OK) return st;
        CK(cudaMemcpyAsync(P.lfac, g.data(), g.size() * 4, cudaMemcpyHostToDevice, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        const float *c0 = P.lfac;
        P.ls = l.hd;
        P.ls.kx = c0;
        P.ls.mx = c0 + 3 * nn[0];
        P.ls.ky = c0 + 6 * nn[0];
        P.ls.my = c0 + 6 * nn[0] + 3 * nn[1];
        P.ls.kz = c0 + 6 * nn[0] + 6 * nn[1];
        P.ls.mz = c0 + 6 * nn[0] + 6 * nn[1] + 3 * nn[2];
      }
    }
  }
  // coarsest-level fast diagonalisation data
  const LevelDev &c = P.L.back().d;
  std::vector<float> Vx, Vy, Vz;
  std::vector<double> lx, ly, lz;
  double cw[4] = {c.wm, c.wx, c.wy, c.wz};
  if (hybrid) {
    axis_eig_tri(c.nx, HK[0], HM[0], Vx, lx);
    axis_eig_tri(c.ny, HK[1], HM[1], Vy, ly);
    if (!batch_z) axis_eig_tri(c.nz, HK[2], HM[2], Vz, lz);
    cw[0] = w[0];
    cw[1] = w[1];
    cw[2] = w[2];
    cw[3] = batch_z ? 0.0 : w[3];
  } else {
    axis_eig(c.nx, c.sx, c.lx, Vx, lx);
    axis_eig(c.ny, c.sy, c.ly, Vy, ly);
    if (!batch_z) axis_eig(c.nz, c.sz, c.lz, Vz, lz);
  }
  const int dz = batch_z ? 1 : c.nz;
  std::vector<double> D((size_t)c.nx * c.ny * dz);
  double dmax = 0.0;
  for (int k = 0; k < dz; ++k)
    for (int j = 0; j < c.ny; ++j)
      for (int i = 0; i < c.nx; ++i) {
        double v = cw[1] * lx[i] + cw[2] * ly[j] + (batch_z ? 0.0 : cw[3] * lz[k]) + cw[0];
        D[((size_t)k * c.ny + j) * c.nx + i] = v;
        dmax = std::fmax(dmax, std::fabs(v));
      }
  std::vector<float> Dinv(D.size());
  for (size_t q = 0; q < D.size(); ++q)  // pseudo-inverse: the constant mode of AD is dropped
    Dinv[q] = (D[q] > 1e-9 * dmax) ? (float)(1.0 / D[q]) : 0.f;
  int st;
  if ((st = dalloc(s, &P.Vx, Vx.size())) != GD_OK) return st;
  if ((st = dalloc(s, &P.Vy, Vy.size())) != GD_OK) return st;
  if (!batch_z && (st = dalloc(s, &P.Vz, Vz.size())) != GD_OK) return st;
  if ((st = dalloc(s, &P.Dinv, Dinv.size())) != GD_OK) return st;
  CK(cudaMemcpyAsync(P.Vx, Vx.data(), Vx.size() * 4, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(P.Vy, Vy.data(), Vy.size() * 4, cudaMemcpyHostToDevice, s->stream));
  if (!batch_z) CK(cudaMemcpyAsync(P.Vz, Vz.data(), Vz.size() * 4, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(P.Dinv, Dinv.data(), Dinv.size() * 4, cudaMemcpyHostToDevice, s->stream));
  CK(cudaStreamSynchronize(s->stream));  // host vectors go out of scope
  P.valid = true;
  return GD_OK;
}

// ---- kernel wrappers with launch accounting ----
// One red-black sweep of level l (x -> t, then the pointers swap), with the
// optional fusions: prolong (x += P x_{l+1} first), restrict (the residual
// summed into level l+1's b afterwards), sum (block sums of the output into
// scalars[S_E]).  Levels whose arrays TMA cannot address run the plain
// kernels with the fused steps as separate passes.
int sweep(gd_stack *s, int li, bool zero_in, bool prolong, bool restrict_, bool sum_e) {
  std::vector<Level> &LV = s->cur->L;
  Level &l = LV[li];
  Level *C = (prolong || restrict_) ? &LV[li + 1] : nullptr;
  const bool fine = li == 0;
  int nb = 0;
  double *part = nullptr;
  if (sum_e) {
    const int gx = (l.d.nx + 63) / 64, gy = (l.d.ny + 15) / 16;
    int st = ensure_partials(s, gx * gy * l.d.nz);
    if (st != GD_OK) return st;
    part = s->partials;
  }
  ZSweepArgs a;
  std::memset(&a, 0, sizeof a);
  a.L = l.d;
  a.xout = l.t;
  a.partials = part;
  a.err = s->scalars + S_ERR;
  if (C) {
    a.xc = C->x;
    a.ncx = C->d.nx;
    a.ncy = C->d.ny;
    a.fx = l.fx;
    a.fy = l.fy;
    a.fz = l.fz;
    a.bc = C->b;
  }
  const bool tma = !s->no_tma && zmarch_usable(l.d, l.esz);
  const int esz_c = C ? C->esz : 4;
  if (!tma && l.esz != 4) {
    set_err(s, "a bfloat16 level needs the TMA kernels");
    return GD_ERR_UNSUPPORTED;
  }
  bool swept = false;
  if (tma) {
    cudaError_t e;
    {
      ProfScope ps(s, fine ? P_SWEEP_FINE : P_SWEEP_COARSE,
                   (double)l.n * l.esz * (zero_in ? 2.0 : 3.0) + (prolong ? (double)esz_c * C->n : 0.0));
      e = launch_zsweep(a, l.x, l.b, zero_in, prolong, sum_e, l.esz, esz_c, &nb, s->stream);
      if (e == cudaErrorNotSupported) {
        s->launches -= 1;
        ps.bytes = 0;
        cudaGetLastError();
      }
    }
    if (e == cudaSuccess) swept = true;
    else if (e != cudaErrorNotSupported) {
      set_err(s, "TMA sweep launch failed: %s", cudaGetErrorString(e));
      return GD_ERR_CUDA;
    }
  }
  if (!swept) {
    if (prolong) {
      ProfScope ps(s, P_PROLONG, (double)l.n * 8.0 + (double)C->n * 4.0);
      CK(launch_prolong_add(l.d, l.fx, l.fy, l.fz, C->x, l.x, s->stream));
    }
    ProfScope ps(s, fine ? P_SWEEP_FINE : P_SWEEP_COARSE, (double)l.n * (zero_in ? 8.0 : 12.0));
    CK(launch_rb_sweep(l.d, l.x, l.b, l.t, zero_in, part, &nb, s->stream));
  }
  if (restrict_) {
    // residual of the relaxed iterate (now in l.t) down-sampled into C->b
    cudaError_t e = cudaErrorNotSupported;
    if (tma) {
      ProfScope ps(s, P_RESTRICT, (double)l.n * 2.0 * l.esz + (double)C->n * esz_c);
      e = launch_zrestrict(a, l.t, l.b, l.esz, esz_c, s->stream);
      if (e == cudaErrorNotSupported) {
        s->launches -= 1;
        ps.bytes = 0;
        cudaGetLastError();
      }
    }
    if (e == cudaErrorNotSupported) {
      ProfScope ps(s, P_RESTRICT, (double)l.n * 8.0 + (double)C->n * 4.0);
      e = launch_residual_restrict(l.d, l.t, l.b, l.fx, l.fy, l.fz, C->b, s->stream);
    }
    if (e != cudaSuccess) {
      set_err(s, "restriction launch failed: %s", cudaGetErrorString(e));
      return GD_ERR_CUDA;
    }
  }
  std::swap(l.x, l.t);
  if (sum_e) {
    ProfScope ps(s, P_REDUCE, (double)nb * S_NUM * 8.0);
    CK(launch_reduce(s->partials, nb, s->scalars, S_E, S_E + 1, 0, s->stream));
  }
  return GD_OK;
}

int coarsest_solve(gd_stack *s, Level &l) {
  Plan &P = *s->cur;
  ProfScope ps(s, P_COARSEST, (double)l.n * 4.0 * (P.batch_z ? 8.0 : 12.0));
  CK(launch_fdm(l.d.nx, l.d.ny, l.d.nz, P.Vx, P.Vy, P.Vz, P.Dinv, P.batch_z, l.b, l.x, l.t,
                s->stream));
  s->launches += P.batch_z ? 3 : 5;
  return GD_OK;
}

// One V(nu1, nu2) cycle of the Hybrid discretisation: red-black sweeps of
// the 6-point fine level, eight-colour sweeps of the 27-point Galerkin
// levels, first-order B-spline transfers as separate passes.
int vcycle_hybrid(gd_stack *s, int nu1, int nu2, bool zero_init, bool sum_e) {
  std::vector<Level> &L = s->cur->L;
  const int nl = (int)L.size();
  const bool six0 = s->disc == GD_DISC_HYBRID;  // the fine level is 6-point (Hybrid) or 27-point (Linear)
  int st;
  if (nl == 1) {
    if ((st = coarsest_solve(s, L[0])) != GD_OK) return st;
    if (six0 && sum_e && (st = sweep(s, 0, false, false, false, true)) != GD_OK) return st;
    return GD_OK;
  }
  auto gs = [&](Level &v) -> int {
    // out of place into the level's second buffer (free during sweeps),
    // then the two swap, as the 6-point sweeps do
    ProfScope ps(s, P_SWEEP_COARSE, (double)v.n * 12.0);
    CK(launch_h_gsf(v.hd, v.x, v.t, v.b, s->stream));
    s->launches += h_gsf_launches(v.hd) - 1;
    std::swap(v.x, v.t);
    return GD_OK;
  };
  for (int l = 0; l < nl - 1; ++l) {
    Level &v = L[l], &c = L[l + 1];
    if (l == 0 && six0) {
      for (int k = 0; k < nu1; ++k)
        if ((st = sweep(s, 0, zero_init && k == 0, false, false, false)) != GD_OK) return st;
    } else {
      if (l > 0 || zero_init) {
        ProfScope ps(s, P_SWEEP_COARSE, (double)v.n * 4.0);
        CK(launch_fill(v.x, v.n, 0.f, s->stream));
      }
      for (int k = 0; k < nu1; ++k)
        if ((st = gs(v)) != GD_OK) return st;
    }
    if (v.fz && !v.fx && !v.fy && v.hd.wz != 0.f && v.d.nz > 1) {
      // halved along z only: residual and restriction in one z-march
      ProfScope ps(s, P_RESTRICT, (double)v.n * 8.0 + (double)c.n * 4.0);
      CK(launch_h_resid_rz(v.hd, l == 0 && six0, v.x, v.b, c.b, c.d.nz, s->stream));
    } else {
      {
        ProfScope ps(s, P_RESTRICT, (double)v.n * 12.0);
        CK(launch_h_resid(v.hd, l == 0 && six0, v.x, v.b, v.t, s->stream));
      }
      {
        ProfScope ps(s, P_RESTRICT, (double)v.n * 4.0 + (double)c.n * 4.0);
        CK(launch_h_restrict(v.d.nx, v.d.ny, v.d.nz, v.fx, v.fy, v.fz, c.d.nx, c.d.ny, c.d.nz, v.t, c.b,
                             s->stream));
      }
    }
  }
  if ((st = coarsest_solve(s, L[nl - 1])) != GD_OK) return st;
  for (int l = nl - 2; l >= 0; --l) {
    Level &v = L[l], &c = L[l + 1];
    {
      ProfScope ps(s, P_PROLONG, (double)v.n * 8.0 + (double)c.n * 4.0);
      CK(launch_h_prolong(v.d.nx, v.d.ny, v.d.nz, v.fx, v.fy, v.fz, c.d.nx, c.d.ny, c.d.nz, c.x, v.x,
                          s->stream));
    }
    if (l == 0 && six0) {
      for (int k = 0; k < nu2; ++k)
        if ((st = sweep(s, 0, false, false, false, sum_e && k == nu2 - 1)) != GD_OK) return st;
    } else {
      for (int k = 0; k < nu2; ++k)
        if ((st = gs(v)) != GD_OK) return st;
    }
  }
  return GD_OK;
}

// One V(nu1,nu2) cycle on level 0's (x, b).  zero_init: level 0's x starts at
// zero (correction form).  sum_e: the last fine sweep also sums its output
// into scalars[S_E].  The last pre-sweep of a level carries the residual and
// its down-sampling; the first post-sweep carries the up-sampled correction.
int vcycle(gd_stack *s, int nu1, int nu2, bool zero_init, bool sum_e) {
  if (s->disc != GD_DISC_CONSTANT) return vcycle_hybrid(s, nu1, nu2, zero_init, sum_e);
  std::vector<Level> &L = s->cur->L;
  const int nl = (int)L.size();
  int st;
  if (nl == 1) {
    // the fine level is the coarsest: x = A^-1 b directly (whatever x was);
    // when the sum of x is wanted, one relaxation sweep (which leaves the
    // exact solution unchanged up to rounding) computes it
    if ((st = coarsest_solve(s, L[0])) != GD_OK) return st;
    if (sum_e && (st = sweep(s, 0, false, false, false, true)) != GD_OK) return st;
    return GD_OK;
  }
  for (int l = 0; l < nl - 1; ++l) {
    const bool zi = (l > 0) || zero_init;
    for (int k = 0; k < nu1; ++k)
      if ((st = sweep(s, l, zi && k == 0, false, k == nu1 - 1, false)) != GD_OK) return st;
  }
  if ((st = coarsest_solve(s, L[nl - 1])) != GD_OK) return st;
  for (int l = nl - 2; l >= 0; --l) {
    for (int k = 0; k < nu2; ++k)
      if ((st = sweep(s, l, false, k == 0, false, sum_e && l == 0 && k == nu2 - 1)) != GD_OK)
        return st;
  }
  return GD_OK;
}

// One V-cycle, replayed from a captured graph when possible.  The first cycle
// with a given shape runs directly (it also performs any lazy allocation),
// and is then captured on a private stream without executing.
int vcycle_run(gd_stack *s, int nu1, int nu2, bool zero_init, bool sum_e) {
  if (s->no_graph) return vcycle(s, nu1, nu2, zero_init, sum_e);
  Plan &P = *s->cur;
  for (auto &gp : P.graphs) {
    VGraph &g = *gp;
    if (g.nu1 == nu1 && g.nu2 == nu2 && g.zero_init == zero_init &&
        g.sum_e == sum_e && g.prof == s->prof_on) {
      if (!g.usable) return vcycle(s, nu1, nu2, zero_init, sum_e);
      CK(cudaGraphLaunch(g.exec, s->stream));
      s->launches += g.launches;
      if (g.prof) s->replayed.push_back(&g);
      return GD_OK;
    }
  }
  const size_t r_direct = s->recs.size();
  int st = vcycle(s, nu1, nu2, zero_init, sum_e);
  if (st != GD_OK) return st;
  std::unique_ptr<VGraph> gp(new VGraph);
  VGraph &g = *gp;
  g.nu1 = nu1;
  g.nu2 = nu2;
  g.zero_init = zero_init;
  g.sum_e = sum_e;
  g.prof = s->prof_on;
  if (!s->cap_stream) CK(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
  // the capture creates no events: take them from the pool
  if (s->prof_on) {
    const size_t need = 2 * (s->recs.size() - r_direct) + 16;
    while (s->ev_pool.size() < need) {
      cudaEvent_t e = nullptr;
      CK(cudaEventCreate(&e));
      s->ev_pool.push_back(e);
    }
  }
  std::vector<float *> saved;
  for (auto &l : P.L) {
    saved.push_back(l.x);
    saved.push_back(l.t);
  }
  cudaStream_t user = s->stream;
  const size_t rec0 = s->recs.size();
  const long long l0 = s->launches;
  s->stream = s->cap_stream;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    s->capturing = true;
    st = vcycle(s, nu1, nu2, zero_init, sum_e);
    s->capturing = false;
    e = cudaStreamEndCapture(s->cap_stream, &graph);
  }
  s->stream = user;
  g.launches = s->launches - l0;
  s->launches = l0;
  g.recs.assign(s->recs.begin() + rec0, s->recs.end());
  s->recs.resize(rec0);
  bool same = true;
  size_t k = 0;
  for (auto &l : P.L) {
    same = same && l.x == saved[k] && l.t == saved[k + 1];
    l.x = saved[k];
    l.t = saved[k + 1];
    k += 2;
  }
  if (e == cudaSuccess && st == GD_OK && same && graph)
    g.usable = cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();  // a failed capture leaves an error behind: fall back to direct launches
  if (!g.usable) release_recs(s, g.recs);
  P.graphs.push_back(std::move(gp));
  return GD_OK;
}

// One outer pass.  esz_e: element size of the correction read and the
// residual written (the fine level's storage).  With h_out the reduced sums
// are read back, and *rmax_out (if given) gets max |r|.
int outer_pass(gd_stack *s, OuterArgs a, int rhs_mode, double *h_out /* [S_NUM] */, int esz_e = 4,
               float *rmax_out = nullptr) {
  a.nx = s->nx;
  a.ny = s->ny;
  a.nz = s->nz;
  a.scalars = s->scalars;
  a.inv_n = 1.0 / ((double)s->nx * s->ny * s->nz);
  const size_t n = (size_t)s->nx * s->ny * s->nz;
  int dev = 0, sms = 152, st;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if ((st = ensure_partials(s, sms * 8 + 64)) != GD_OK) return st;
  if ((st = ensure_partials(s, zouter_max_blocks(s->nx, s->ny, s->nz))) != GD_OK) return st;
  a.partials = s->partials;
  if (a.e_scale == 0.f) a.e_scale = 1.f;
  if (a.r_scale == 0.f) a.r_scale = 1.f;
  a.rmax = reinterpret_cast<unsigned *>(s->scalars + S_RMAX);
  CK(cudaMemsetAsync(s->scalars + S_RMAX, 0, sizeof(double), s->stream));
  double bytes = (4.0 * (1 + (a.xl_in ? 1 : 0) + (a.xh_out ? 1 : 0) + (a.xl_out ? 1 : 0) +
                         (rhs_mode == RHS_SP ? 2 : 1)) +
                  (double)esz_e * ((a.e ? 1 : 0) + (a.r_out ? 1 : 0))) *
                 (double)n;
  int nb = 0;
  {
    ProfScope ps(s, P_OUTER, bytes);
    cudaError_t e = s->no_tma ? cudaErrorNotSupported
                              : launch_zouter(a, rhs_mode, esz_e, s->scalars + S_ERR, &nb, s->stream);
    if (e == cudaErrorNotSupported && esz_e == 4) {
      cudaGetLastError();
      e = launch_outer(a, rhs_mode, &nb, s->stream);
    }
    if (e != cudaSuccess) {
      set_err(s, "outer pass launch failed: %s", cudaGetErrorString(e));
      return GD_ERR_CUDA;
    }
  }
  {
    ProfScope ps(s, P_REDUCE, (double)nb * S_NUM * 8.0);
    CK(launch_reduce(s->partials, nb, s->scalars, S_RR, S_I0 + 1, 0, s->stream));
  }
  if (h_out) {
    CK(cudaMemcpyAsync(s->h_scalars, s->scalars, 8 * sizeof(double), cudaMemcpyDeviceToHost,
                       s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (!s->replayed.empty()) prof_collect_graphs(s);
    std::memcpy(h_out, s->h_scalars, S_NUM * sizeof(double));
    if (rmax_out) {
      unsigned u;
      std::memcpy(&u, s->h_scalars + S_RMAX, sizeof u);
      std::memcpy(rmax_out, &u, sizeof u);
    }
    if (s->h_scalars[S_ERR] != 0.0) {
      const int code = (int)s->h_scalars[S_ERR];
      if (code == 1) {
        set_err(s, "a kernel's bounded wait for its TMA loads gave up");
        return GD_ERR_TIMEOUT;
      }
      set_err(s, "a TMA kernel refused to start (preflight code %d: 2 smem base, 3 tensor "
                 "map, 4 smem size)", code);
      return GD_ERR_CUDA;
    }
  }
  return GD_OK;
}

int ensure_common(gd_stack *s) {
  if (!s->scalars) {
    if (cudaMalloc((void **)&s->scalars, 8 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return GD_ERR_OOM;
    }
    cudaMemsetAsync(s->scalars, 0, 8 * sizeof(double), s->stream);
  }
  if (!s->h_scalars) {
    if (cudaMallocHost((void **)&s->h_scalars, 8 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return GD_ERR_OOM;
    }
  }
  return GD_OK;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// A device array of another GPU: the stack's kernels would read it from the
// wrong device (without peer access, an illegal address), so it is refused.
bool on_other_device(const gd_stack *s, const void *p) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return s->device >= 0 && at.type == cudaMemoryTypeDevice && at.device != s->device;
}

// Device view of a caller array: device pointers pass through; host arrays
// are copied (if `in`) into staging buffer `slot`.
// A host array in pinned memory the GPU can address (allocated by
// cudaHostAlloc, or registered and mapped): its device address, else
// nullptr.
float *mapped_host(const void *p) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? static_cast<float *>(at.devicePointer) : nullptr;
}
// n floats between a host array and the device: pinned host memory moves
// with the wide copy kernel (many loads in flight across the CPU-GPU link:
// faster than one copy-engine transfer there), other host memory with
// cudaMemcpyAsync.
cudaError_t copy_h2d(float *dst, const float *src, size_t n, cudaStream_t st) {
  if (const float *m = mapped_host(src)) return launch_copy_wide(dst, m, n, st);
  return cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyHostToDevice, st);
}
cudaError_t copy_d2h(float *dst, const float *src, size_t n, cudaStream_t st) {
  if (float *m = mapped_host(dst)) return launch_copy_wide(m, src, n, st);
  return cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyDeviceToHost, st);
}

int resolve(gd_stack *s, const float *p, bool in, int slot, float **dev) {
  if (!p) {
    *dev = nullptr;
    return GD_OK;
  }
  if (on_other_device(s, p)) {
    set_err(s, "array %p lives on another device than the stack's (device %d)", (const void *)p,
            s->device);
    return GD_ERR_INVALID_ARG;
  }
  if (is_device_ptr(p)) {
    *dev = const_cast<float *>(p);
    return GD_OK;
  }
  const size_t n = (size_t)s->nx * s->ny * s->nz;
  if (!s->stage[slot]) {
    int st = dalloc(s, &s->stage[slot], n);
    if (st != GD_OK) return st;
  }
  if (in) {
    CK(copy_h2d(s->stage[slot], p, n, s->stream));
  }
  *dev = s->stage[slot];
  return GD_OK;
}

bool finite_nonneg(double v) { return std::isfinite(v) && v >= 0.0; }

// w = hi + lo with hi = fl32(w): the weights of the outer residual as float pairs
void split(double w, float &hi, float &lo) {
  hi = (float)w;
  lo = (float)(w - (double)hi);
}

void set_weights(OuterArgs &a, double bx, double by, double bz, double alpha, double rbx,
                 double rby, double ralpha) {
  split(bx, a.bx, a.bx_lo);
  split(by, a.by, a.by_lo);
  split(bz, a.bz, a.bz_lo);
  split(alpha, a.alpha, a.alpha_lo);
  split(rbx, a.rbx, a.rbx_lo);
  split(rby, a.rby, a.rby_lo);
  split(ralpha, a.ralpha, a.ralpha_lo);
}

int check_ctl(gd_stack *s, const gd_solve_ctl *ctl, gd_solve_ctl *out) {
  gd_solve_ctl c = {20, 1e-6, 2, 2, 16, 0};
  if (ctl) c = *ctl;
  if (c.coarsest_xy == 0) c.coarsest_xy = 16;
  if (c.max_cycles < 0 || c.nu1 < 1 || c.nu1 > 8 || c.nu2 < 1 || c.nu2 > 8 ||
      c.coarsest_xy < 2 || c.coarsest_xy > 4096 || !(c.rel_tol >= 0.0) ||
      (c.rel_tol <= 0.0 && c.max_cycles <= 0)) {
    set_err(s, "invalid solve control (max_cycles %d, rel_tol %g, nu1 %d, nu2 %d, coarsest_xy %d)",
            c.max_cycles, c.rel_tol, c.nu1, c.nu2, c.coarsest_xy);
    return GD_ERR_INVALID_ARG;
  }
  *out = c;
  return GD_OK;
}

void rep_init(gd_report *rep) {
  if (!rep) return;
  std::memset(rep, 0, sizeof(*rep));
  rep->rel_residual_out = NAN;
  rep->rel_residual = NAN;
  rep->rho_per_cycle = NAN;
}

// Solve one of the two systems with iterative refinement on the float pair.
// The Linear discretisation's driver: the right-hand side once as a float
// pair, then V-cycles on the correction with the float-pair iterate updated
// (TwoSum) and its residual evaluated in compensated float arithmetic after
// each; AD keeps the plain
// sum of I0 by a constant shift of the output (the constant is A's null
// space, so the shift changes no residual).
int solve_linear(gd_stack *s, int system, const float *I0h, const float *I1h, float *outh, double w[4],
                 const gd_solve_ctl *ctl_in, const float *x0h, gd_report *rep) {
  rep_init(rep);
  gd_solve_ctl ctl;
  int st = check_ctl(s, ctl_in, &ctl);
  if (st != GD_OK) return report(rep, st);
  if ((st = ensure_common(s)) != GD_OK) return report(rep, st);
  const size_t n = (size_t)s->nx * s->ny * s->nz;
  float *I0 = nullptr, *I1 = nullptr, *out = nullptr, *x0 = nullptr;
  const bool out_host = !is_device_ptr(outh);
  if ((st = resolve(s, I0h, true, 0, &I0)) != GD_OK) return report(rep, st);
  if (system == GD_SYSTEM_SP && (st = resolve(s, I1h, true, 1, &I1)) != GD_OK) return report(rep, st);
  const bool generic = system == SYS_GENERIC;
  if ((st = resolve(s, outh, false, 2, &out)) != GD_OK) return report(rep, st);
  if (x0h && (st = resolve(s, x0h, true, 3, &x0)) != GD_OK) return report(rep, st);
  const bool uncoupled = system == GD_SYSTEM_SP || (generic && w[3] == 0.0);
  if ((st = plan_build(s, w, uncoupled, ctl.coarsest_xy, GD_PREC_FP32)) != GD_OK) return report(rep, st);
  Plan &P = *s->cur;
  Level &F = P.L[0];
  if (rep) rep->levels = (int)P.L.size();
  // float pair of the iterate (xh2, xl1) and of the right-hand side (xl2, out)
  if (!s->xh2 && (st = dalloc(s, &s->xh2, n)) != GD_OK) return report(rep, st);
  if (!s->xl1 && (st = dalloc(s, &s->xl1, n)) != GD_OK) return report(rep, st);
  if (!s->xl2 && (st = dalloc(s, &s->xl2, n)) != GD_OK) return report(rep, st);
  if (!s->lbh && (st = dalloc(s, &s->lbh, n)) != GD_OK) return report(rep, st);
  float *xh = s->xh2, *xl = s->xl1, *bh = s->lbh, *bl = s->xl2;
  LinW lw;
  if (system == GD_SYSTEM_SP)
    lw = LinW{w[1], w[2], 0.0, w[0], 1.0, 1.0, w[0]};
  else if (generic)
    lw = LinW{w[1], w[2], uncoupled ? 0.0 : w[3], w[0], 0.0, 0.0, 0.0};
  else
    lw = LinW{w[1], w[2], w[3], 0.0, w[1], w[2], 0.0};
  const HLevelDev &L0 = P.ls;
  {
    // the kernels sum over the integer-scaled factors: divide each weight by
    // the scales of the mass factors in its term
    const double sx = P.lscale[0], sy = P.lscale[1], sz = P.lscale[2];
    lw.ax /= sy * sz;
    lw.ay /= sx * sz;
    lw.az /= sx * sy;
    lw.am /= sx * sy * sz;
    lw.gx /= sy * sz;
    lw.gy /= sx * sz;
    lw.gm /= sx * sy * sz;
  }
  const int mean_fix = system == GD_SYSTEM_AD;
  int nb = 0;
  {
    ProfScope ps(s, P_OUTER, (double)n * 16.0);
    if (generic) {
      CK(launch_copy(bh, I0, n, s->stream));
      CK(launch_fill(bl, n, 0.f, s->stream));
    } else {
      CK(launch_l_rhs(L0, lw, I0, I1, bh, bl, s->stream));
    }
  }
  {
    ProfScope ps(s, P_COPY, (double)n * 8.0);
    const float *start = x0 ? x0 : (system == GD_SYSTEM_SP ? I0 : nullptr);
    if (start)
      CK(launch_copy(xh, start, n, s->stream));
    else
      CK(launch_fill(xh, n, 0.f, s->stream));
    CK(launch_fill(xl, n, 0.f, s->stream));
  }
  if ((st = ensure_partials(s, std::max(linear_grid((long long)n), linear_zmax_blocks(L0)) + 8)) != GD_OK)
    return report(rep, st);
  double sum_i0 = 0.0;
  auto reduce_read = [&](int lo, int hi, double *outv) -> int {
    CK(launch_reduce(s->partials, nb, s->scalars, lo, hi, 0, s->stream));
    CK(cudaMemcpyAsync(s->h_scalars, s->scalars, 8 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    for (int k = lo; k < hi; ++k) outv[k] = s->h_scalars[k];
    return GD_OK;
  };
  double hs[S_NUM] = {0, 0, 0, 0, 0};
  if (mean_fix) {
    CK(launch_l_sum((long long)n, I0, s->partials, S_I0, &nb, s->stream));
    if ((st = reduce_read(S_I0, S_I0 + 1, hs)) != GD_OK) return report(rep, st);
    sum_i0 = hs[S_I0];
  }
  auto residual = [&](double *rel_out, double *bnorm_out) -> int {
    {
      ProfScope ps(s, P_OUTER, (double)n * 20.0);
      CK(launch_l_resid(L0, lw, bh, bl, xh, xl, F.b, s->partials, &nb, s->stream));
    }
    int r = reduce_read(S_RR, S_BB + 1, hs);
    if (r != GD_OK) return r;
    *bnorm_out = std::sqrt(hs[S_BB]);
    *rel_out = std::sqrt(hs[S_RR]) / (*bnorm_out > 0.0 ? *bnorm_out : 1.0);
    return GD_OK;
  };
  double rel = 0.0, bnorm = 0.0;
  if ((st = residual(&rel, &bnorm)) != GD_OK) return report(rep, st);
  const double rel0 = rel;
  if (rep) {
    rep->rhs_norm = bnorm;
    rep->history[0] = rel;
  }
  int cycles = 0, status = GD_OK;
  std::vector<double> hist(1, rel);
  double sum_x = 0.0;
  bool have_sum_x = false;
  while (!(rel <= ctl.rel_tol)) {
    if (cycles >= ctl.max_cycles) {
      status = GD_ERR_NOT_CONVERGED;
      break;
    }
    if ((st = vcycle_run(s, ctl.nu1, ctl.nu2, true, false)) != GD_OK) return report(rep, st);
    {
      ProfScope ps(s, P_OUTER, (double)n * 20.0);
      CK(launch_l_update((long long)n, F.x, xh, xl, s->partials, &nb, s->stream));
    }
    if (mean_fix) {
      if ((st = reduce_read(S_X, S_X + 1, hs)) != GD_OK) return report(rep, st);
      sum_x = hs[S_X];
      have_sum_x = true;
    }
    if ((st = residual(&rel, &bnorm)) != GD_OK) return report(rep, st);
    ++cycles;
    hist.push_back(rel);
    if (rep && cycles < GD_HISTORY) rep->history[cycles] = rel;
    if (!std::isfinite(rel) || rel > 1e3 * std::fmax(rel0, 1e-300)) {
      status = GD_ERR_DIVERGED;
      break;
    }
    if (cycles >= 4 && rel > 0.7 * hist[cycles - 3] && rel > ctl.rel_tol) {
      status = GD_ERR_NOT_CONVERGED;
      break;
    }
  }
  double shift = 0.0;
  if (mean_fix) {
    if (!have_sum_x) {
      CK(launch_l_sum((long long)n, xh, s->partials, S_X, &nb, s->stream));
      if ((st = reduce_read(S_X, S_X + 1, hs)) != GD_OK) return report(rep, st);
      sum_x = hs[S_X];  // the low words are zero before the first update
    }
    shift = (sum_i0 - sum_x) / (double)n;
  }
  {
    ProfScope ps(s, P_COPY, (double)n * 12.0);
    CK(launch_l_final((long long)n, xh, xl, shift, out, s->stream));
  }
  if (rep) {
    rep->cycles = cycles;
    rep->rel_residual = rel;
    rep->rho_per_cycle = cycles > 0 && rel0 > 0 ? std::pow(rel / rel0, 1.0 / cycles) : NAN;
  }
  if (out_host) CK(copy_d2h(outh, out, n, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (s->prof_on) prof_collect(s);
  return report(rep, status);
}

int solve(gd_stack *s, int system, const float *I0h, const float *I1h, float *outh, double w[4],
          const gd_solve_ctl *ctl_in, const float *x0h, gd_report *rep) {
  if (s->disc == GD_DISC_LINEAR) return solve_linear(s, system, I0h, I1h, outh, w, ctl_in, x0h, rep);
  rep_init(rep);
  gd_solve_ctl ctl;
  int st = check_ctl(s, ctl_in, &ctl);
  if (st != GD_OK) return report(rep, st);
  if ((st = ensure_common(s)) != GD_OK) return report(rep, st);
  const size_t n = (size_t)s->nx * s->ny * s->nz;
  // device views
  float *I0 = nullptr, *I1 = nullptr, *out = nullptr, *x0 = nullptr;
  const bool out_host = !is_device_ptr(outh);
  if ((st = resolve(s, I0h, true, 0, &I0)) != GD_OK) return report(rep, st);
  if (system == GD_SYSTEM_SP && (st = resolve(s, I1h, true, 1, &I1)) != GD_OK) return report(rep, st);
  const bool generic = system == SYS_GENERIC;  // I0 holds the explicit right-hand side
  if ((st = resolve(s, outh, x0h == outh, 2, &out)) != GD_OK) return report(rep, st);
  if (x0h && x0h != outh && (st = resolve(s, x0h, true, 3, &x0)) != GD_OK) return report(rep, st);
  if (x0h == outh) x0 = out;
  const bool uncoupled = system == GD_SYSTEM_SP || (generic && w[3] == 0.0);
  if ((st = plan_build(s, w, uncoupled, ctl.coarsest_xy, s->prec)) != GD_OK)
    return report(rep, st);
  Plan &P = *s->cur;
  if (!s->xh2 && (st = dalloc(s, &s->xh2, n)) != GD_OK) return report(rep, st);
  if (!s->xl1 && (st = dalloc(s, &s->xl1, n)) != GD_OK) return report(rep, st);
  if (!s->xl2 && (st = dalloc(s, &s->xl2, n)) != GD_OK) return report(rep, st);
  if (rep) rep->levels = (int)P.L.size();

  // initial iterate in `out`
  // Default start.  AD: zero (relative residual 1; starting from I0 leaves
  // the removed inter-slice variation, several times the right-hand side,
  // and costs a cycle).  SP: I0, whose residual alpha (I1 - I0) is a few
  // thousandths of the right-hand side on EM stacks (from I1 about half of
  // it remains).
  const float *start = x0 ? x0 : (system == GD_SYSTEM_SP ? I0 : nullptr);
  if (!start) {
    ProfScope ps(s, P_COPY, (double)n * 4.0);
    CK(launch_fill(out, n, 0.f, s->stream));
  } else if (start != out) {
    ProfScope ps(s, P_COPY, (double)n * 8.0);
    CK(launch_copy(out, start, n, s->stream));
  }
  OuterArgs a;
  std::memset(&a, 0, sizeof a);
  if (system == GD_SYSTEM_SP)
    set_weights(a, w[1], w[2], 0.0, w[0], 1.0, 1.0, w[0]);
  else if (generic)
    set_weights(a, w[1], w[2], w[3], w[0], 0.0, 0.0, 0.0);
  else
    set_weights(a, w[1], w[2], w[3], 0.0, w[1], w[2], 0.0);
  a.I0 = I0;
  a.I1 = I1;
  a.b = generic ? I0 : nullptr;
  const int rhs = generic ? RHS_EXPLICIT : (system == GD_SYSTEM_SP ? RHS_SP : RHS_AD);
  const int mean_fix = system == GD_SYSTEM_AD;
  Level &F = P.L[0];
  const int esz = F.esz;  // storage of the correction solve (4, or 2 when mixed)

  double h[S_NUM];
  // bfloat16 storage keeps float32's exponent range: no scaling is needed
  // (the scale hooks of the outer pass stay at 1)
  auto run_pass = [&](OuterArgs &pa) -> int {
    pa.e_scale = 1.f;
    pa.r_scale = 1.f;
    return outer_pass(s, pa, rhs, h, esz);
  };

  // initial residual
  a.xh_in = out;
  a.r_out = F.b;
  if ((st = run_pass(a)) != GD_OK) return report(rep, st);
  const double bnorm = std::sqrt(h[S_BB]);
  const double denom = bnorm > 0.0 ? bnorm : 1.0;
  double rel = std::sqrt(h[S_RR]) / denom;
  const double rel0 = rel;
  if (rep) {
    rep->rhs_norm = bnorm;
    rep->history[0] = rel;
  }
  // float-pair buffers: pass k reads pair c and writes pair 1-c; the low
  // part of the starting iterate is zero and is not read
  float *H[2] = {out, s->xh2};
  float *Lo[2] = {s->xl2, s->xl1};
  int c = 0;
  bool lo_zero = true;
  int cycles = 0;
  int status = GD_OK;
  std::vector<double> hist(1, rel);
  bool exact = false;
  auto update = [&](const float *e) -> int {
    // Plain FP32 passes while the residual is large: their rounding error
    // (~1e-7 of the local terms) and the dropped low word of the iterate are
    // then far below the residual.  From 1e-4 on (and from then on always)
    // the iterate is a float pair and the residual is evaluated exactly.
    if (rel < 1e-4) exact = true;
    a.accurate = exact ? 1 : 0;
    a.xh_in = H[c];
    a.xl_in = lo_zero ? nullptr : Lo[c];
    a.e = e;
    a.mean_fix = mean_fix;
    a.xh_out = H[1 - c];
    a.xl_out = exact ? Lo[1 - c] : nullptr;
    a.r_out = F.b;
    int r = run_pass(a);
    c = 1 - c;
    if (exact) lo_zero = false;
    return r;
  };
  while (!(rel <= ctl.rel_tol)) {
    if (cycles >= ctl.max_cycles) {
      status = GD_ERR_NOT_CONVERGED;
      break;
    }
    if ((st = vcycle_run(s, ctl.nu1, ctl.nu2, true, mean_fix)) != GD_OK) return report(rep, st);
    if ((st = update(F.x)) != GD_OK) return report(rep, st);
    ++cycles;
    rel = std::sqrt(h[S_RR]) / denom;
    hist.push_back(rel);
    if (rep && cycles < GD_HISTORY) rep->history[cycles] = rel;
    if (!std::isfinite(rel) || rel > 1e3 * std::fmax(rel0, 1e-300)) {
      status = GD_ERR_DIVERGED;
      break;
    }
    // stall: less than a 30% gain over the last three cycles (precision floor)
    if (cycles >= 4 && rel > 0.7 * hist[cycles - 3] && rel > ctl.rel_tol) {
      status = GD_ERR_NOT_CONVERGED;
      break;
    }
  }
  if (mean_fix && cycles == 0) {
    // no cycle ran: still move the start's mean to mean(I0)
    CK(cudaMemsetAsync(F.x, 0, n * esz, s->stream));
    CK(cudaMemsetAsync(s->scalars + S_E, 0, sizeof(double), s->stream));
    if ((st = update(F.x)) != GD_OK) return report(rep, st);
    rel = std::sqrt(h[S_RR]) / denom;
  }
  float *cur_h = H[c];
  // result into `out`
  if (cur_h != out) {
    ProfScope ps(s, P_COPY, (double)n * 8.0);
    CK(launch_copy(out, cur_h, n, s->stream));
  }
  if (rep) {
    rep->cycles = cycles;
    rep->rel_residual = rel;
    rep->rho_per_cycle = cycles > 0 && rel0 > 0 ? std::pow(rel / rel0, 1.0 / cycles) : NAN;
  }
  if (rep && (ctl.flags & GD_FLAG_REPORT_OUTPUT_RESIDUAL)) {
    OuterArgs b2 = a;
    b2.xh_in = out;
    b2.xl_in = nullptr;
    b2.e = nullptr;
    b2.xh_out = b2.xl_out = nullptr;
    b2.r_out = nullptr;
    b2.mean_fix = 0;
    b2.accurate = 1;
    if ((st = outer_pass(s, b2, rhs, h)) != GD_OK) return report(rep, st);
    rep->rel_residual_out = std::sqrt(h[S_RR]) / denom;
  }
  if (out_host) {
    CK(copy_d2h(outh, out, n, s->stream));
  }
  CK(cudaStreamSynchronize(s->stream));
  if (s->prof_on) prof_collect(s);
  return report(rep, status);
}

bool weights_ok(const gd_weights &w) {
  return finite_nonneg(w.alpha) && finite_nonneg(w.beta_x) && finite_nonneg(w.beta_y) &&
         finite_nonneg(w.beta_z);
}

}  // namespace

extern "C" {

int gd_version(void) { return 1; }

const char *gd_status_string(int st) {
  switch (st) {
    case GD_OK: return "ok";
    case GD_ERR_INVALID_ARG: return "invalid argument";
    case GD_ERR_UNSUPPORTED: return "unsupported";
    case GD_ERR_OOM: return "out of memory";
    case GD_ERR_CUDA: return "CUDA error";
    case GD_ERR_NOT_CONVERGED: return "not converged";
    case GD_ERR_DIVERGED: return "diverged";
    case GD_ERR_TIMEOUT: return "timeout";
    default: return "unknown status";
  }
}

const char *gd_last_error(gd_stack *s) { return s ? s->err.c_str() : "null stack"; }

int gd_stack_create(gd_stack **out, int nx, int ny, int nz, int bc, int disc, int prec,
                    void *cuda_stream) {
  if (!out) return GD_ERR_INVALID_ARG;
  *out = nullptr;
  if (nx < 2 || ny < 2 || nz < 1) return GD_ERR_INVALID_ARG;
  if ((double)nx * ny * nz > 9.0e18 / 64) return GD_ERR_INVALID_ARG;
  if (bc != GD_BC_NEUMANN) return GD_ERR_UNSUPPORTED;
  if (disc != GD_DISC_CONSTANT && disc != GD_DISC_HYBRID && disc != GD_DISC_LINEAR) return GD_ERR_INVALID_ARG;
  if (prec != GD_PREC_FP32 && prec != GD_PREC_MIXED) return GD_ERR_INVALID_ARG;
  if (disc != GD_DISC_CONSTANT && prec != GD_PREC_FP32) return GD_ERR_UNSUPPORTED;
  gd_stack *s = new (std::nothrow) gd_stack();
  if (!s) return GD_ERR_OOM;
  s->nx = nx;
  s->ny = ny;
  s->nz = nz;
  s->bc = bc;
  s->disc = disc;
  s->prec = prec;
  s->stream = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&s->device) != cudaSuccess) {  // no device yet: creation needs none
    cudaGetLastError();
    s->device = -1;
  }
  const char *nt = std::getenv("GD_DISABLE_TMA");
  s->no_tma = nt && nt[0] && std::strcmp(nt, "0") != 0;
  const char *ng = std::getenv("GD_DISABLE_GRAPHS");
  s->no_graph = ng && ng[0] && std::strcmp(ng, "0") != 0;
  const char *fa = std::getenv("GD_FAIL_ALLOC_AFTER");
  if (fa && fa[0]) s->fail_alloc_after = std::atoll(fa);
  *out = s;
  return GD_OK;
}

int gd_destroy(gd_stack *s) {
  if (!s) return GD_OK;
  cudaStreamSynchronize(s->stream);
  if (!s->replayed.empty()) prof_collect_graphs(s);
  for (auto &p : s->plans) plan_free(s, *p);
  s->plans.clear();
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  dfree(s->f_x);
  dfree(s->f_b);
  dfree(s->f_t);
  dfree(s->xh2);
  dfree(s->xl1);
  dfree(s->xl2);
  dfree(s->lbh);
  dfree(s->i1);
  for (auto &p : s->stage) dfree(p);
  if (s->partials) cudaFree(s->partials);
  if (s->scalars) cudaFree(s->scalars);
  if (s->h_scalars) cudaFreeHost(s->h_scalars);
  for (auto &r : s->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : s->ev_pool) cudaEventDestroy(e);
  delete s;
  return GD_OK;
}

int gd_diffuse_z(gd_stack *s, const float *I0, float *I1, gd_weights w, const gd_solve_ctl *ctl,
                 const float *x0, gd_report *rep) {
  rep_init(rep);
  if (!s || !I0 || !I1) return report(rep, GD_ERR_INVALID_ARG);
  if (I0 == I1) {
    set_err(s, "I1 must not alias I0");
    return report(rep, GD_ERR_INVALID_ARG);
  }
  if (!weights_ok(w) || !(w.beta_z > 0.0) || !(w.beta_x + w.beta_y > 0.0)) {
    set_err(s, "AD needs finite weights with beta_x, beta_y >= 0, beta_x + beta_y > 0, beta_z > 0");
    return report(rep, GD_ERR_INVALID_ARG);
  }
  double wv[4] = {0.0, w.beta_x, w.beta_y, w.beta_z};
  return solve(s, GD_SYSTEM_AD, I0, nullptr, I1, wv, ctl, x0, rep);
}

int gd_screened_poisson_slices(gd_stack *s, const float *I0, const float *I1, float *I2,
                               double alpha, const gd_solve_ctl *ctl, const float *x0,
                               gd_report *rep) {
  rep_init(rep);
  if (!s || !I0 || !I1 || !I2) return report(rep, GD_ERR_INVALID_ARG);
  if (I2 == I0 || I2 == I1) {
    set_err(s, "I2 must alias neither I0 nor I1");
    return report(rep, GD_ERR_INVALID_ARG);
  }
  if (!std::isfinite(alpha) || !(alpha > 0.0)) {
    set_err(s, "SP needs a finite alpha > 0");
    return report(rep, GD_ERR_INVALID_ARG);
  }
  double wv[4] = {alpha, 1.0, 1.0, 0.0};
  return solve(s, GD_SYSTEM_SP, I0, I1, I2, wv, ctl, x0, rep);
}

int gd_ad_then_sp(gd_stack *s, const float *I0h, float *I2h, gd_weights w_ad, double alpha,
                  const gd_solve_ctl *ctl_ad, const gd_solve_ctl *ctl_sp, float *I1h, gd_report *rep_ad,
                  gd_report *rep_sp) {
  rep_init(rep_ad);
  rep_init(rep_sp);
  if (!s || !I0h || !I2h || I0h == I2h || (I1h && (I1h == I0h || I1h == I2h))) {
    if (s) set_err(s, "gd_ad_then_sp needs I0 and I2 (and the optional I1) as distinct arrays");
    report(rep_ad, GD_ERR_INVALID_ARG);
    return report(rep_sp, GD_ERR_INVALID_ARG);
  }
  if (!std::isfinite(alpha) || !(alpha > 0.0)) {
    set_err(s, "SP needs a finite alpha > 0");
    report(rep_ad, GD_ERR_INVALID_ARG);
    return report(rep_sp, GD_ERR_INVALID_ARG);
  }
  int st = ensure_common(s);
  if (st != GD_OK) return report(rep_sp, report(rep_ad, st));
  const size_t n = (size_t)s->nx * s->ny * s->nz;
  // I0 on the device once (host arrays are staged here, so both solves find
  // a device pointer and copy nothing); I1 stays on the device
  float *I0 = nullptr;
  if ((st = resolve(s, I0h, true, 0, &I0)) != GD_OK) return report(rep_sp, report(rep_ad, st));
  float *I1 = nullptr;
  const bool i1_dev = I1h && is_device_ptr(I1h);
  if (i1_dev) {
    I1 = I1h;
  } else {
    if (!s->i1 && (st = dalloc(s, &s->i1, n)) != GD_OK) return report(rep_sp, report(rep_ad, st));
    I1 = s->i1;
  }
  st = gd_diffuse_z(s, I0, I1, w_ad, ctl_ad, nullptr, rep_ad);
  if (st != GD_OK && st != GD_ERR_NOT_CONVERGED) return report(rep_sp, st);
  const int st_ad = st;
  st = gd_screened_poisson_slices(s, I0, I1, I2h, alpha, ctl_sp, nullptr, rep_sp);
  if (st != GD_OK && st != GD_ERR_NOT_CONVERGED) return st;
  if (I1h && !i1_dev) {
    CK(copy_d2h(I1h, I1, n, s->stream));
    CK(cudaStreamSynchronize(s->stream));
  }
  return st != GD_OK ? st : st_ad;
}

int gd_selftest_wait(unsigned polls) {
  if (polls == 0 || polls > (1u << 24)) return GD_ERR_INVALID_ARG;
  const int r = zmarch_wait_selftest(polls, nullptr);
  if (r < 0) return GD_ERR_CUDA;
  return r == 1 ? GD_ERR_TIMEOUT : GD_OK;
}

int gd_screened_poisson(gd_stack *s, gd_weights w, const float *b, float *x, const gd_solve_ctl *ctl,
                        const float *x0, gd_report *rep) {
  rep_init(rep);
  if (!s || !b || !x) return report(rep, GD_ERR_INVALID_ARG);
  if (x == b) {
    set_err(s, "x must not alias b");
    return report(rep, GD_ERR_INVALID_ARG);
  }
  if (!weights_ok(w) || !(w.alpha > 0.0)) {
    set_err(s, "the general solve needs finite weights >= 0 and alpha > 0");
    return report(rep, GD_ERR_INVALID_ARG);
  }
  double wv[4] = {w.alpha, w.beta_x, w.beta_y, w.beta_z};
  return solve(s, SYS_GENERIC, b, nullptr, x, wv, ctl, x0, rep);
}

int gd_npr_rhs(gd_stack *s, const float *I0h, float *bh, gd_weights w, double lambda, double sigma) {
  if (!s || !I0h || !bh || I0h == bh || !weights_ok(w) || !std::isfinite(lambda) ||
      !std::isfinite(sigma) || !(sigma > 0.0))
    return GD_ERR_INVALID_ARG;
  int st;
  if ((st = ensure_common(s)) != GD_OK) return st;
  const size_t n = (size_t)s->nx * s->ny * s->nz;
  float *I0 = nullptr, *b = nullptr;
  const bool b_host = !is_device_ptr(bh);
  if ((st = resolve(s, I0h, true, 0, &I0)) != GD_OK) return st;
  if ((st = resolve(s, bh, false, 2, &b)) != GD_OK) return st;
  {
    ProfScope ps(s, P_COPY, (double)n * 8.0);
    CK(launch_npr_rhs(I0, b, s->nx, s->ny, s->nz, w.alpha, w.beta_x, w.beta_y, w.beta_z, lambda, sigma,
                      s->stream));
  }
  if (b_host) CK(copy_d2h(bh, b, n, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (s->prof_on) prof_collect(s);
  return GD_OK;
}

int gd_vcycle(gd_stack *s, int system, gd_weights w, const float *bh, float *xh, int ncycles,
              gd_report *rep) {
  rep_init(rep);
  if (!s || !bh || !xh || ncycles < 0 || bh == xh) return report(rep, GD_ERR_INVALID_ARG);
  if (!weights_ok(w)) return report(rep, GD_ERR_INVALID_ARG);
  if (s->disc == GD_DISC_LINEAR) {
    set_err(s, "gd_vcycle evaluates the 6-point fine operator; the Linear discretisation solves "
               "through gd_diffuse_z / gd_screened_poisson_slices / gd_screened_poisson");
    return report(rep, GD_ERR_UNSUPPORTED);
  }
  if (system == GD_SYSTEM_AD) {
    if (!(w.beta_z > 0.0)) return report(rep, GD_ERR_INVALID_ARG);
  } else if (system == GD_SYSTEM_SP) {
    if (w.beta_z != 0.0 || !(w.alpha > 0.0)) return report(rep, GD_ERR_INVALID_ARG);
  } else {
    return report(rep, GD_ERR_INVALID_ARG);
  }
  int st;
  if ((st = ensure_common(s)) != GD_OK) return report(rep, st);
  const size_t n = (size_t)s->nx * s->ny * s->nz;
  float *b = nullptr, *x = nullptr;
  const bool x_host = !is_device_ptr(xh);
  if ((st = resolve(s, bh, true, 0, &b)) != GD_OK) return report(rep, st);
  if ((st = resolve(s, xh, true, 2, &x)) != GD_OK) return report(rep, st);
  double wv[4] = {w.alpha, w.beta_x, w.beta_y, w.beta_z};
  if ((st = plan_build(s, wv, system == GD_SYSTEM_SP, 16)) != GD_OK) return report(rep, st);
  Level &F = s->cur->L[0];
  OuterArgs a;
  std::memset(&a, 0, sizeof a);
  set_weights(a, w.beta_x, w.beta_y, w.beta_z, w.alpha, 0.0, 0.0, 0.0);
  a.accurate = 1;
  a.b = b;
  a.xh_in = x;
  double h[S_NUM];
  if ((st = outer_pass(s, a, RHS_EXPLICIT, h)) != GD_OK) return report(rep, st);
  const double bnorm = std::sqrt(h[S_BB]);
  const double denom = bnorm > 0.0 ? bnorm : 1.0;
  const double rel0 = std::sqrt(h[S_RR]) / denom;
  // run the cycles directly on the caller's x (level 0 borrows x and b)
  float *wsx = F.x, *wst = F.t, *wsb = F.b;
  F.x = x;
  F.b = b;
  F.t = wst;
  for (int c = 0; c < ncycles && st == GD_OK; ++c) {
    st = vcycle(s, 2, 2, false, false);
    if (st == GD_OK && F.x != x) {  // odd number of ping-pong swaps: move back
      ProfScope ps(s, P_COPY, (double)n * 8.0);
      if (launch_copy(x, F.x, n, s->stream) != cudaSuccess) st = GD_ERR_CUDA;
      F.x = x;
      F.t = wst;
    }
  }
  F.x = wsx;
  F.t = wst;
  F.b = wsb;
  if (st != GD_OK) return report(rep, st);
  if ((st = outer_pass(s, a, RHS_EXPLICIT, h)) != GD_OK) return report(rep, st);
  const double rel = std::sqrt(h[S_RR]) / denom;
  if (rep) {
    rep->cycles = ncycles;
    rep->levels = (int)s->cur->L.size();
    rep->rhs_norm = bnorm;
    rep->rel_residual = rel;
    rep->history[0] = rel0;
    rep->history[1] = rel;
    rep->rho_per_cycle = ncycles > 0 && rel0 > 0 ? std::pow(rel / rel0, 1.0 / ncycles) : NAN;
  }
  if (x_host) CK(copy_d2h(xh, x, n, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (s->prof_on) prof_collect(s);
  return report(rep, GD_OK);
}

int gd_residual(gd_stack *s, int system, gd_weights w, const float *I0h, const float *I1h,
                const float *xh, double *rel) {
  if (!s || !I0h || !xh || !rel) return GD_ERR_INVALID_ARG;
  if (system != GD_SYSTEM_AD && system != GD_SYSTEM_SP) return GD_ERR_INVALID_ARG;
  if (system == GD_SYSTEM_SP && (!I1h || !(w.alpha > 0.0))) return GD_ERR_INVALID_ARG;
  if (!weights_ok(w)) return GD_ERR_INVALID_ARG;
  if (s->disc == GD_DISC_LINEAR) {
    set_err(s, "gd_residual evaluates the 6-point operator, not the Linear discretisation's");
    return GD_ERR_UNSUPPORTED;
  }
  int st;
  if ((st = ensure_common(s)) != GD_OK) return st;
  float *I0 = nullptr, *I1 = nullptr, *x = nullptr;
  if ((st = resolve(s, I0h, true, 0, &I0)) != GD_OK) return st;
  if (system == GD_SYSTEM_SP && (st = resolve(s, I1h, true, 1, &I1)) != GD_OK) return st;
  if ((st = resolve(s, xh, true, 3, &x)) != GD_OK) return st;
  OuterArgs a;
  std::memset(&a, 0, sizeof a);
  const bool sp = system == GD_SYSTEM_SP;
  if (sp)
    set_weights(a, 1.0, 1.0, 0.0, w.alpha, 1.0, 1.0, w.alpha);
  else
    set_weights(a, w.beta_x, w.beta_y, w.beta_z, 0.0, w.beta_x, w.beta_y, 0.0);
  a.I0 = I0;
  a.I1 = I1;
  a.xh_in = x;
  a.accurate = 1;
  double h[S_NUM];
  if ((st = outer_pass(s, a, sp ? RHS_SP : RHS_AD, h)) != GD_OK) return st;
  const double bn = std::sqrt(h[S_BB]);
  *rel = std::sqrt(h[S_RR]) / (bn > 0 ? bn : 1.0);
  return GD_OK;
}

int gd_smooth(gd_stack *s, gd_weights w, const float *bh, float *xh, int nsweeps) {
  if (!s || !bh || !xh || nsweeps < 0 || bh == xh || !weights_ok(w)) return GD_ERR_INVALID_ARG;
  if (s->disc == GD_DISC_LINEAR) {
    set_err(s, "gd_smooth relaxes the 6-point operator, not the Linear discretisation's");
    return GD_ERR_UNSUPPORTED;
  }
  int st;
  if ((st = ensure_common(s)) != GD_OK) return st;
  const size_t n = (size_t)s->nx * s->ny * s->nz;
  float *b = nullptr, *x = nullptr;
  const bool x_host = !is_device_ptr(xh);
  if ((st = resolve(s, bh, true, 0, &b)) != GD_OK) return st;
  if ((st = resolve(s, xh, true, 2, &x)) != GD_OK) return st;
  // a one-level plan of the given weights, borrowing the caller's arrays
  Plan *saved = s->cur;
  Plan tmp_plan;
  s->cur = &tmp_plan;
  Level l;
  l.d = LevelDev{s->nx, s->ny, s->nz, 1, 1, 1, 1, 1, 1, (float)w.beta_x, (float)w.beta_y,
                 (float)w.beta_z, (float)w.alpha};
  l.n = n;
  l.b = b;
  l.x = x;
  // the sweep's second array is the stack's fine workspace (allocated once,
  // shared with the solves, which never run at the same time on one stack)
  if (!s->f_t && (st = dalloc(s, &s->f_t, n)) != GD_OK) {
    s->cur = saved;
    return st;
  }
  l.t = s->f_t;
  tmp_plan.L.push_back(l);
  for (int k = 0; k < nsweeps && st == GD_OK; ++k) st = sweep(s, 0, false, false, false, false);
  Level &lr = tmp_plan.L[0];
  if (st == GD_OK && lr.x != x) {
    ProfScope ps(s, P_COPY, (double)n * 8.0);
    if (launch_copy(x, lr.x, n, s->stream) != cudaSuccess) st = GD_ERR_CUDA;
  }
  if (st == GD_OK && x_host)
    if (copy_d2h(xh, x, n, s->stream) != cudaSuccess)
      st = GD_ERR_CUDA;
  cudaStreamSynchronize(s->stream);
  tmp_plan.L.clear();
  s->cur = saved;
  if (s->prof_on) prof_collect(s);
  return st;
}

int gd_profile_enable(gd_stack *s, int on) {
  if (!s) return GD_ERR_INVALID_ARG;
  cudaStreamSynchronize(s->stream);
  if (!s->replayed.empty()) prof_collect_graphs(s);
  if (!on) prof_collect(s);
  s->prof_on = on != 0;
  return GD_OK;
}

int gd_profile_reset(gd_stack *s) {
  if (!s) return GD_ERR_INVALID_ARG;
  prof_collect(s);
  for (int k = 0; k < P_NUM; ++k) {
    s->prof_launches[k] = 0;
    s->prof_ms[k] = 0;
    s->prof_bytes[k] = 0;
  }
  return GD_OK;
}

int gd_profile_query(gd_stack *s, int k, char *name, int name_len, long long *launches,
                     double *ms, double *bytes) {
  if (!s || k < 0 || k >= P_NUM) return GD_ERR_INVALID_ARG;
  prof_collect(s);
  if (name && name_len > 0) {
    std::strncpy(name, kProfNames[k], (size_t)name_len - 1);
    name[name_len - 1] = 0;
  }
  if (launches) *launches = s->prof_launches[k];
  if (ms) *ms = s->prof_ms[k];
  if (bytes) *bytes = s->prof_bytes[k];
  return GD_OK;
}

long long gd_launch_count(gd_stack *s) { return s ? s->launches : -1; }

int gd_level_count(gd_stack *s) { return s && s->cur ? (int)s->cur->L.size() : 0; }

int gd_level_info(gd_stack *s, int level, int *info, double *weights) {
  if (!s || !s->cur || level < 0 || level >= (int)s->cur->L.size() || !info || !weights)
    return GD_ERR_INVALID_ARG;
  if (s->disc != GD_DISC_CONSTANT) {
    set_err(s, "level inspection describes the Constant discretisation's 6-point levels");
    return GD_ERR_UNSUPPORTED;
  }
  const Level &l = s->cur->L[level];
  const int v[10] = {l.d.nx, l.d.ny, l.d.nz, l.d.sx, l.d.sy, l.d.sz, l.d.lx, l.d.ly, l.d.lz, l.esz};
  for (int k = 0; k < 10; ++k) info[k] = v[k];
  weights[0] = l.d.wx;
  weights[1] = l.d.wy;
  weights[2] = l.d.wz;
  weights[3] = l.d.wm;
  return GD_OK;
}

int gd_level_fetch(gd_stack *s, int level, int which, float *dst) {
  if (!s || !s->cur || level < 1 || level >= (int)s->cur->L.size() || (which != 0 && which != 1) || !dst)
    return GD_ERR_INVALID_ARG;
  if (s->disc != GD_DISC_CONSTANT) {
    set_err(s, "level inspection describes the Constant discretisation's 6-point levels");
    return GD_ERR_UNSUPPORTED;
  }
  if (on_other_device(s, dst)) return GD_ERR_INVALID_ARG;
  const Level &l = s->cur->L[level];
  const float *src = which == 0 ? l.x : l.b;
  if (!src) return GD_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return GD_ERR_CUDA;
  const bool dev = is_device_ptr(dst);
  if (l.esz == 4) {
    return cudaMemcpy(dst, src, l.n * sizeof(float), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost) ==
                   cudaSuccess
               ? GD_OK
               : GD_ERR_CUDA;
  }
  // bfloat16 storage: widen on the host (a bfloat16 is the high half of a float32)
  std::vector<uint16_t> h(l.n);
  std::vector<float> f(l.n);
  if (cudaMemcpy(h.data(), src, l.n * sizeof(uint16_t), cudaMemcpyDeviceToHost) != cudaSuccess) return GD_ERR_CUDA;
  for (size_t i = 0; i < l.n; ++i) {
    const uint32_t u = (uint32_t)h[i] << 16;
    std::memcpy(&f[i], &u, sizeof u);
  }
  return cudaMemcpy(dst, f.data(), l.n * sizeof(float), dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost) ==
                 cudaSuccess
             ? GD_OK
             : GD_ERR_CUDA;
}

}  // extern "C"
