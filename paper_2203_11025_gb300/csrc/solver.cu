// libhelm driver: handle, workspace, V-cycle orchestration, coarsest GMRES,
// restarted FGMRES with one CUDA graph per restart cycle, and the C ABI
// declared in include/helm.h.
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/helm.h"
#include "helm_internal.cuh"
#include "block_ls.h"
#include "unet_api.h"
#include "unet_internal.cuh"

namespace {
thread_local std::string g_err;
}  // namespace

namespace helm {
void set_error(const std::string& s) { g_err = s; }
}  // namespace helm

#define HCHECK(call)                                                                          \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      g_err = std::string(#call) + ": " + cudaGetErrorString(e_);                             \
      return HELM_ECUDA;                                                                      \
    }                                                                                         \
  } while (0)
#define HLAUNCH()                                                                             \
  do {                                                                                        \
    cudaError_t e_ = cudaGetLastError();                                                      \
    if (e_ != cudaSuccess) {                                                                  \
      g_err = std::string("kernel launch: ") + cudaGetErrorString(e_);                        \
      return HELM_ECUDA;                                                                      \
    }                                                                                         \
  } while (0)
#define HTRY(call)               \
  do {                           \
    int r_ = (call);             \
    if (r_ < 0) return r_;       \
  } while (0)

using namespace helm;

namespace {

// A device arena: one cudaMalloc carved into 256-byte aligned pieces.
struct Arena {
  char* base = nullptr;
  size_t size = 0, used = 0;
  void* take(size_t bytes) {
    size_t off = (used + 255) & ~(size_t)255;
    if (off + bytes > size) return nullptr;
    used = off + bytes;
    return base + off;
  }
};

// Workspace for one real type T (float: solver; double: FP64 checking runs).
struct Work {
  int cap = 0;               // right-hand sides the buffers hold
  int m = 0;                 // FGMRES restart length the buffers hold
  Arena arena;
  std::vector<void*> F, E, T1, T2;   // per level: restricted rhs, coarse correction, two scratch vectors
  void* CV = nullptr;                // coarsest GMRES basis [(mc+1)][rhs][Nc]
  ArnoldiState cst{};                // coarsest GMRES state
  void* V = nullptr;                 // FGMRES basis [(m+1)][rhs][N]
  void* Z = nullptr;                 // FGMRES preconditioned vectors [m][rhs][N]
  ArnoldiState fst{};
  SolveState ss{};
  double2* bx = nullptr;             // staging for HOST_IO: b and x (FP64) [rhs][N] each
  double2* xx = nullptr;
  void* S0 = nullptr;                // two fine-grid scratch vectors for the U-Net preconditioners
  void* S1 = nullptr;
  int* maxit_rhs = nullptr;          // per right-hand-side iteration caps (pair generator)
};

// A captured cycle bakes in every device pointer it touches: the solver's work arena
// (graphs are dropped when it is reallocated), b and x, and the network's weights and
// workspace -- identified by the network's unique id and workspace generation rather
// than its address, which a later network may reuse.
struct GraphKey {
  int dtype, precond, nrhs, m, maxit;
  const void* b;
  const void* x;
  unsigned long long net[4];
  bool operator<(const GraphKey& o) const {
    return std::tie(dtype, precond, nrhs, m, maxit, b, x, net[0], net[1], net[2], net[3]) <
           std::tie(o.dtype, o.precond, o.nrhs, o.m, o.maxit, o.b, o.x, o.net[0], o.net[1], o.net[2], o.net[3]);
  }
};
constexpr size_t kMaxGraphs = 64;   // cached cycles (older ones belong to released buffers)

}  // namespace

struct helm_ctx {
  helm_desc d{};
  int device = 0, nsm = 148;
  std::vector<Level> L;
  void* level_mem = nullptr;
  Work w32, w64;
  cudaStream_t own = nullptr;        // stream that graphs are captured on and launched from
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int* h_done = nullptr;             // pinned host mirror of done flags
  std::map<GraphKey, cudaGraphExec_t> graphs;
  std::map<GraphKey, long long> graph_kernels;  // kernel nodes per captured cycle
  float* gam0 = nullptr;             // absorbing-layer attenuation on the fine grid (float32)
  bool fused_coarse = true;          // one-launch coarsest GMRES when the grid fits in shared memory
  bool cluster_coarse = true;        // cluster-resident coarsest GMRES when the grid fits
  // tile tuner: segment height of the fused cycle kernels per (kernel, level, nrhs), chosen
  // by timing the candidates once (see tune_cycle_tiles); absent: chosen by occupancy
  std::map<std::tuple<int, int, int>, int> seg;
  int nmedia = 1;                    // media held (a batch of problems of one grid size)
  int rpp = 0;                       // right-hand sides per medium (0: one medium for every one)
};

namespace {

size_t level_points(const helm_ctx* c, int l) { return (size_t)c->L[l].nx * c->L[l].ny; }

void free_work(Work& W) {
  if (W.arena.base) cudaFree(W.arena.base);
  W = Work();
}

void drop_graphs(helm_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
  c->graph_kernels.clear();
}

template <typename T> Work& work_of(helm_ctx* c);
template <> Work& work_of<float>(helm_ctx* c) { return c->w32; }
template <> Work& work_of<double>(helm_ctx* c) { return c->w64; }

// (Re)allocate the workspace of type T for `nrhs` right-hand sides and restart m.
template <typename T>
int ensure_work(helm_ctx* c, int nrhs, int m) {
  Work& W = work_of<T>(c);
  if (W.cap >= nrhs && W.m >= m) return HELM_OK;
  nrhs = std::max(nrhs, W.cap);
  m = std::max(m, std::max(W.m, c->d.coarse_its));
  drop_graphs(c);
  free_work(W);
  const int L = c->d.levels;
  const size_t es = sizeof(typename vec2<T>::type);
  const size_t N0 = level_points(c, 0), Nc = level_points(c, L - 1);
  const int mc = c->d.coarse_its;
  const int nbmax = 4096;
  const int mcap = c->nsm * 8 + 8;   // >= every vec_blocks() count
  auto st_bytes = [&](int mm) {
    return (size_t)nrhs * ((size_t)(mm + 1) * mm * 16 * 2 + mm * 8 + mm * 16 + (mm + 1) * 16 + mm * 16 + 8 * 3 +
                           4 * 4 + (size_t)nbmax * 16 + (size_t)kProjMax * 16 +
                           (size_t)(kProjMax + 1) * mcap * 16) + 256 * 20;
  };
  size_t total = 0;
  for (int l = 0; l < L; ++l) total += 4 * (nrhs * level_points(c, l) * es + 256);
  total += (size_t)(mc + 1) * nrhs * Nc * es + 256;
  total += (size_t)(2 * m + 1) * nrhs * N0 * es + 512;
  total += 2 * (size_t)nrhs * N0 * 16 + 512;
  total += 2 * ((size_t)nrhs * N0 * es + 256) + (size_t)nrhs * 4 + 256;
  total += st_bytes(mc) + st_bytes(m) + (size_t)nrhs * 64 + 4096;
  void* mem = nullptr;
  if (cudaMalloc(&mem, total) != cudaSuccess) {
    cudaGetLastError();
    g_err = "workspace allocation of " + std::to_string(total) + " bytes failed";
    return HELM_ENOMEM;
  }
  W.arena.base = (char*)mem;
  W.arena.size = total;
  W.cap = nrhs;
  W.m = m;
  W.F.assign(L, nullptr); W.E.assign(L, nullptr); W.T1.assign(L, nullptr); W.T2.assign(L, nullptr);
  for (int l = 0; l < L; ++l) {
    size_t b = nrhs * level_points(c, l) * es;
    W.F[l] = W.arena.take(b); W.E[l] = W.arena.take(b); W.T1[l] = W.arena.take(b); W.T2[l] = W.arena.take(b);
  }
  W.CV = W.arena.take((size_t)(mc + 1) * nrhs * Nc * es);
  W.V = W.arena.take((size_t)(m + 1) * nrhs * N0 * es);
  W.Z = W.arena.take((size_t)m * nrhs * N0 * es);
  W.bx = (double2*)W.arena.take((size_t)nrhs * N0 * 16);
  W.xx = (double2*)W.arena.take((size_t)nrhs * N0 * 16);
  W.S0 = W.arena.take((size_t)nrhs * N0 * es);
  W.S1 = W.arena.take((size_t)nrhs * N0 * es);
  W.maxit_rhs = (int*)W.arena.take((size_t)nrhs * 4);
  auto make_st = [&](ArnoldiState& st, int mm) {
    st.m = mm;
    st.nbmax = nbmax;
    st.H = (double2*)W.arena.take((size_t)nrhs * (mm + 1) * mm * 16);
    st.R = (double2*)W.arena.take((size_t)nrhs * (mm + 1) * mm * 16);
    st.cs = (double*)W.arena.take((size_t)nrhs * mm * 8);
    st.sn = (double2*)W.arena.take((size_t)nrhs * mm * 16);
    st.g = (double2*)W.arena.take((size_t)nrhs * (mm + 1) * 16);
    st.y = (double2*)W.arena.take((size_t)nrhs * mm * 16);
    st.beta = (double*)W.arena.take((size_t)nrhs * 8);
    st.est = (double*)W.arena.take((size_t)nrhs * 8);
    st.tol_abs = (double*)W.arena.take((size_t)nrhs * 8);
    st.active = (int*)W.arena.take((size_t)nrhs * 4);
    st.k = (int*)W.arena.take((size_t)nrhs * 4);
    st.kmax = (int*)W.arena.take((size_t)nrhs * 4);
    st.counter = (int*)W.arena.take((size_t)nrhs * 4);
    st.part = (double2*)W.arena.take((size_t)nrhs * nbmax * 16);
    st.proj = (double2*)W.arena.take((size_t)nrhs * kProjMax * 16);
    st.mcap = mcap;
    st.mpart = (double2*)W.arena.take((size_t)nrhs * (kProjMax + 1) * mcap * 16);
  };
  make_st(W.cst, mc);
  make_st(W.fst, m);
  W.ss.bnorm = (double*)W.arena.take((size_t)nrhs * 8);
  W.ss.relres = (double*)W.arena.take((size_t)nrhs * 8);
  W.ss.done = (int*)W.arena.take((size_t)nrhs * 4);
  W.ss.iters = (int*)W.arena.take((size_t)nrhs * 4);
  W.ss.status = (int*)W.arena.take((size_t)nrhs * 4);
  W.ss.maxit_rhs = nullptr;
  if (!W.ss.status || !W.fst.part || !W.fst.mpart || !W.cst.mpart) {
    g_err = "workspace layout overflow";
    free_work(W);
    return HELM_ENOMEM;
  }
  // zero everything: counters must start at 0, coarse tol_abs = 0 (run all steps)
  HCHECK(cudaMemset(W.arena.base, 0, W.arena.size));
  if (c->h_done) cudaFreeHost(c->h_done);
  HCHECK(cudaMallocHost(&c->h_done, (size_t)nrhs * sizeof(int)));
  return HELM_OK;
}

template <typename T> Op<T> op_on(helm_ctx* c, int level, double beta) {
  return make_op<T>(c->L[level], c->d.omega, c->d.abc_gamma_max, beta);
}

// ---------------------------------------------------------------------------
// Coarsest grid: GMRES(mc) on M D^-1 y = f from 0, x = D^-1 y (Sec. 2.4, 4).
template <typename T>
int coarse_gmres(helm_ctx* c, const void* f, void* out, int nrhs, const int* gate, cudaStream_t s) {
  Work& W = work_of<T>(c);
  const int lc = c->d.levels - 1, mc = c->d.coarse_its;
  const size_t Nc = level_points(c, lc);
  const size_t es = sizeof(typename vec2<T>::type);
  const size_t vstride = (size_t)nrhs * Nc;
  char* CV = (char*)W.CV;
  Op<T> op = op_on<T>(c, lc, c->d.beta);
  if (c->cluster_coarse && launch_coarse_gmres_cluster<T>(op, f, out, nrhs, mc, gate, CV, vstride, s)) {
    HLAUNCH();
    return HELM_OK;
  }
  if (c->fused_coarse && launch_coarse_gmres_fused<T>(op, f, out, CV, vstride, nrhs, mc, gate, s)) {
    HLAUNCH();
    return HELM_OK;
  }
  ArnoldiState& st = W.cst;
  const int nb = vec_blocks(Nc, nrhs, c->nsm);
  launch_start<T>(f, CV, Nc, nrhs, st, nb, gate, s);
  for (int j = 0; j < mc; ++j)
    launch_arnoldi<T>(op, true, CV + (size_t)j * vstride * es, CV, vstride, nrhs, st, j, mc, nb, s);
  launch_backsolve(st, nrhs, nullptr, s);
  launch_combine<T>(CV, vstride, Nc, nrhs, st, &op, out, gate, nb, s);
  HLAUNCH();
  return HELM_OK;
}

// out = V-cycle(v_in, f) on `level` of M (Alg. 1).  v_in == nullptr: zero guess.
// out must not alias f or v_in.
template <typename T>
int vcycle(helm_ctx* c, int level, const void* f, const void* v_in, void* out, int nrhs, const int* gate,
           cudaStream_t s) {
  Work& W = work_of<T>(c);
  const helm_desc& d = c->d;
  if (level == d.levels - 1) return coarse_gmres<T>(c, f, out, nrhs, gate, s);
  const Level& Lv = c->L[level];
  const Op<T> op = op_on<T>(c, level, d.beta);
  const T w = (T)d.jacobi_w;
  const size_t bytes = (size_t)nrhs * level_points(c, level) * sizeof(typename vec2<T>::type);
  void* sa = W.T1[level];
  void* sb = W.T2[level];
  // pre-smoothing: the first sweep from a zero guess stays implicit (fused)
  const void* cur = v_in;
  bool implicit = false;
  int nu1 = d.nu1;
  if (!cur && nu1 >= 1) { implicit = true; --nu1; }
  if (implicit && nu1 > 0) {
    launch_jacobi<T>(op, w, f, nullptr, sa, nrhs, gate, s);
    cur = sa; implicit = false;
    std::swap(sa, sb);
  }
  for (; nu1 > 0; --nu1) {
    launch_jacobi<T>(op, w, f, cur, sa, nrhs, gate, s);
    cur = sa;
    std::swap(sa, sb);
  }
  if (cur == out) {  // only when nu1 == 0 and v_in aliases out
    HCHECK(cudaMemcpyAsync(sa, cur, bytes, cudaMemcpyDeviceToDevice, s));
    cur = sa;
    std::swap(sa, sb);
  }
  // residual, restriction, coarse correction
  void* fc = W.F[level + 1];
  auto seg_of = [&](int kind) {
    auto it = c->seg.find(std::make_tuple(kind, level, nrhs));
    return it == c->seg.end() ? 0 : it->second;
  };
  if (implicit || cur)
    launch_resid_restrict<T>(op, w, f, implicit ? nullptr : cur, fc, nrhs, gate, s, seg_of(0));
  else launch_restrict<T>(Lv.nx, Lv.ny, f, fc, nrhs, gate, s);
  void* ec = W.E[level + 1];
  HTRY(vcycle<T>(c, level + 1, fc, nullptr, ec, nrhs, gate, s));
  const int nxc = c->L[level + 1].nx, nyc = c->L[level + 1].ny;
  // correction and post-smoothing
  if (d.nu2 == 0) {
    if (implicit) launch_jacobi<T>(op, w, f, nullptr, out, nrhs, gate, s);
    else if (cur) HCHECK(cudaMemcpyAsync(out, cur, bytes, cudaMemcpyDeviceToDevice, s));
    else HCHECK(cudaMemsetAsync(out, 0, bytes, s));
    launch_prolong_add<T>(nxc, nyc, Lv.nx, Lv.ny, ec, out, nrhs, gate, s);
  } else {
    int nu2 = d.nu2;
    void* dst = (nu2 == 1) ? out : (sa != cur ? sa : sb);
    launch_prolong_jacobi<T>(op, w, f, implicit ? nullptr : cur, implicit, ec, nxc, nyc, dst, nrhs, gate, s,
                             seg_of(1));
    const void* x = dst;
    for (--nu2; nu2 > 0; --nu2) {
      void* nxt = (nu2 == 1) ? out : (x == sa ? sb : sa);
      launch_jacobi<T>(op, w, f, x, nxt, nrhs, gate, s);
      x = nxt;
    }
  }
  HLAUNCH();
  return HELM_OK;
}

// z = M^-1 v for the chosen preconditioner.
template <typename T>
int precond_apply(helm_ctx* c, int precond, void* net, const void* v, void* z, int nrhs, const int* gate,
                  cudaStream_t s) {
  const size_t bytes = (size_t)nrhs * level_points(c, 0) * sizeof(typename vec2<T>::type);
  switch (precond) {
    case HELM_PREC_NONE:
      HCHECK(cudaMemcpyAsync(z, v, bytes, cudaMemcpyDeviceToDevice, s));
      return HELM_OK;
    case HELM_PREC_V:
      return vcycle<T>(c, 0, v, nullptr, z, nrhs, gate, s);
    case HELM_PREC_JU:
    case HELM_PREC_VU:
      return unet_precond_impl(c, net, precond, v, z, nrhs, (int)sizeof(T), gate, s);
    default:
      g_err = "unknown preconditioner";
      return HELM_EINVAL;
  }
}

// One restart cycle's Arnoldi steps and the update x += Z y (graph-capturable).
template <typename T>
int fgmres_cycle(helm_ctx* c, int precond, void* net, double2* x, int nrhs, int m, cudaStream_t s) {
  Work& W = work_of<T>(c);
  const size_t N = level_points(c, 0);
  const size_t es = sizeof(typename vec2<T>::type);
  const size_t vstride = (size_t)nrhs * N;
  char* V = (char*)W.V;
  char* Z = (char*)W.Z;
  ArnoldiState& st = W.fst;
  const Op<T> A = op_on<T>(c, 0, 0.0);
  const int nb = vec_blocks(N, nrhs, c->nsm);
  launch_scale_v0<T>(V, N, nrhs, st, nb, s);
  for (int j = 0; j < m; ++j) {
    void* vj = V + (size_t)j * vstride * es;
    void* zj = Z + (size_t)j * vstride * es;
    void* w = V + (size_t)(j + 1) * vstride * es;
    HTRY(precond_apply<T>(c, precond, net, vj, zj, nrhs, st.active, s));
    launch_arnoldi<T>(A, false, zj, V, vstride, nrhs, st, j, m, nb, s);
  }
  launch_backsolve(st, nrhs, W.ss.iters, s);
  launch_update_x<T>(Z, vstride, N, nrhs, st, x, nb, s);
  HLAUNCH();
  return HELM_OK;
}

// Tile tuner of the fused cycle kernels (FP32): for every level with a coarser one, time
// each segment height of the column-strip form (4, 8, 16, 32 rows) and the shared-memory
// tile form (-1) on the workspace vectors of nrhs right-hand sides (contents irrelevant)
// and keep the fastest, once per (level, nrhs).  Runs outside graph capture; the choices
// then hold for every captured cycle.
int tune_cycle_tiles(helm_ctx* c, int nrhs, cudaStream_t s) {
  if (c->d.stencil != HELM_STENCIL_5PT) return HELM_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  HCHECK(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) return HELM_OK;
  Work& W = c->w32;
  if (W.cap < nrhs) return HELM_OK;
  cudaEvent_t e0, e1;
  HCHECK(cudaEventCreate(&e0));
  HCHECK(cudaEventCreate(&e1));
  const float w = (float)c->d.jacobi_w;
  for (int l = 0; l + 1 < c->d.levels; ++l) {
    const Op<float> op = op_on<float>(c, l, c->d.beta);
    const int nxc = c->L[l + 1].nx, nyc = c->L[l + 1].ny;
    for (int kind = 0; kind < 2; ++kind) {
      if (c->seg.count(std::make_tuple(kind, l, nrhs))) continue;   // tuned, or set by the caller
      int best = 0;
      float best_ms = 1e30f;
      for (int seg : {4, 8, 16, 32, -1}) {
        auto run = [&] {
          if (kind == 0) launch_resid_restrict<float>(op, w, W.T1[l], nullptr, W.F[l + 1], nrhs, nullptr, s, seg);
          else launch_prolong_jacobi<float>(op, w, W.T1[l], nullptr, true, W.E[l + 1], nxc, nyc, W.T2[l], nrhs,
                                            nullptr, s, seg);
        };
        run();
        HCHECK(cudaEventRecord(e0, s));
        for (int r = 0; r < 3; ++r) run();
        HCHECK(cudaEventRecord(e1, s));
        HCHECK(cudaEventSynchronize(e1));
        float ms = 0;
        HCHECK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) { best_ms = ms; best = seg; }
      }
      c->seg[std::make_tuple(kind, l, nrhs)] = best;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HLAUNCH();
  return HELM_OK;
}

// One FGMRES solve split into phases, so that several handles can interleave their
// restart cycles (fgmres_solve_batch): prepare (workspace, ||b||, network workspace, tile
// tuning, the captured cycle), then per round check (FP64 true residual and the done
// flags, copied to the host) / done / cycle, then finish.
struct FgJob {
  helm_ctx* c = nullptr;
  int precond = 0;
  void* net = nullptr;
  const double2* b = nullptr;
  double2* x = nullptr;
  int nrhs = 0;
  fgmres_opts o{};
  const int* maxit_rhs_host = nullptr;
  cudaStream_t caller = nullptr;
  fgmres_result* res = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long per_cycle = -1;
  int cycles = 0, nb = 0;
  bool finished = false;
};

template <typename T>
int fg_prepare(FgJob& J) {
  helm_ctx* c = J.c;
  const fgmres_opts& o = J.o;
  const int nrhs = J.nrhs, m = o.restart;
  HTRY(ensure_work<T>(c, nrhs, o.restart));
  Work& W = work_of<T>(c);
  if (J.maxit_rhs_host) {
    HCHECK(cudaMemcpyAsync(W.maxit_rhs, J.maxit_rhs_host, nrhs * sizeof(int), cudaMemcpyHostToDevice, J.caller));
    W.ss.maxit_rhs = W.maxit_rhs;
  } else {
    W.ss.maxit_rhs = nullptr;
  }
  const size_t N = level_points(c, 0);
  J.nb = vec_blocks(N, nrhs, c->nsm);
  cudaStream_t s = c->own;
  HCHECK(cudaEventRecord(c->ev_in, J.caller));
  HCHECK(cudaStreamWaitEvent(s, c->ev_in, 0));
  if (o.flags & HELM_FLAG_X0_ZERO) HCHECK(cudaMemsetAsync(J.x, 0, (size_t)nrhs * N * 16, s));
  launch_bnorm(J.b, N, nrhs, W.ss, W.fst, J.nb, o.tol, s);
  HLAUNCH();
  if (J.precond == HELM_PREC_JU || J.precond == HELM_PREC_VU) HTRY(unet_prepare_impl(c, J.net, nrhs));
  if (sizeof(T) == 4 && !(o.flags & HELM_FLAG_NO_GRAPH)) HTRY(tune_cycle_tiles(c, nrhs, s));
  J.exec = nullptr;
  J.per_cycle = -1;
  J.cycles = 0;
  J.finished = false;
  if (!(o.flags & HELM_FLAG_NO_GRAPH)) {
    GraphKey key{(int)sizeof(T), J.precond, nrhs, m, o.maxit, J.b, J.x, {0, 0, 0, 0}};
    if (J.net) unet_graph_ids(J.net, key.net);
    if (J.maxit_rhs_host) key.maxit = -1 - o.maxit;
    if (c->graphs.size() >= kMaxGraphs && !c->graphs.count(key)) drop_graphs(c);
    auto it = c->graphs.find(key);
    if (it != c->graphs.end()) {
      J.exec = it->second;
      J.per_cycle = c->graph_kernels[key];
    } else {
      cudaGraph_t g;
      HCHECK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      int r = fgmres_cycle<T>(c, J.precond, J.net, J.x, nrhs, m, s);
      cudaError_t ce = cudaStreamEndCapture(s, &g);
      if (r < 0) return r;
      if (ce != cudaSuccess) { g_err = std::string("graph capture: ") + cudaGetErrorString(ce); return HELM_ECUDA; }
      size_t nn = 0;
      HCHECK(cudaGraphGetNodes(g, nullptr, &nn));
      std::vector<cudaGraphNode_t> nodes(nn);
      HCHECK(cudaGraphGetNodes(g, nodes.data(), &nn));
      J.per_cycle = 0;
      for (auto nd : nodes) {
        cudaGraphNodeType ty;
        HCHECK(cudaGraphNodeGetType(nd, &ty));
        if (ty == cudaGraphNodeTypeKernel) ++J.per_cycle;
      }
      HCHECK(cudaGraphInstantiate(&J.exec, g, 0));
      cudaGraphDestroy(g);
      c->graphs[key] = J.exec;
      c->graph_kernels[key] = J.per_cycle;
    }
  }
  return HELM_OK;
}

// Enqueue the FP64 true residual of every right-hand side and the copy of the done flags.
template <typename T>
int fg_check(FgJob& J) {
  helm_ctx* c = J.c;
  Work& W = work_of<T>(c);
  const Op<double> A64 = op_on<double>(c, 0, 0.0);
  launch_true_residual<T>(A64, J.b, J.x, W.V, J.nrhs, W.ss, W.fst, J.nb, J.o.maxit, c->own);
  HLAUNCH();
  HCHECK(cudaMemcpyAsync(c->h_done, W.ss.done, (size_t)J.nrhs * sizeof(int), cudaMemcpyDeviceToHost, c->own));
  return HELM_OK;
}

// After the check has completed: true when every right-hand side is done; otherwise the
// next restart cycle is launched.
template <typename T>
int fg_step(FgJob& J, bool* done) {
  helm_ctx* c = J.c;
  HCHECK(cudaStreamSynchronize(c->own));
  bool all = true;
  for (int r = 0; r < J.nrhs; ++r) all = all && c->h_done[r];
  *done = all;
  if (all) return HELM_OK;
  const int max_cycles = J.o.maxit / std::max(1, J.o.restart) + 3 + J.o.maxit;
  if (++J.cycles > max_cycles) { g_err = "FGMRES cycle guard tripped"; return HELM_ECUDA; }
  if (J.exec) HCHECK(cudaGraphLaunch(J.exec, c->own));
  else HTRY(fgmres_cycle<T>(c, J.precond, J.net, J.x, J.nrhs, J.o.restart, c->own));
  return HELM_OK;
}

template <typename T>
int fg_finish(FgJob& J) {
  helm_ctx* c = J.c;
  Work& W = work_of<T>(c);
  cudaStream_t s = c->own;
  const int nrhs = J.nrhs;
  std::vector<int> iters(nrhs), status(nrhs);
  std::vector<double> relres(nrhs);
  HCHECK(cudaMemcpyAsync(iters.data(), W.ss.iters, nrhs * sizeof(int), cudaMemcpyDeviceToHost, s));
  HCHECK(cudaMemcpyAsync(status.data(), W.ss.status, nrhs * sizeof(int), cudaMemcpyDeviceToHost, s));
  HCHECK(cudaMemcpyAsync(relres.data(), W.ss.relres, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
  HCHECK(cudaStreamSynchronize(s));
  HCHECK(cudaEventRecord(c->ev_out, s));
  HCHECK(cudaStreamWaitEvent(J.caller, c->ev_out, 0));
  int st = HELM_OK;
  fgmres_result* res = J.res;
  if (res) {
    res->iters_max = 0;
    res->relres_max = 0;
    res->cycles = J.cycles;
    // bnorm + one true-residual kernel per check + the cycle graphs
    res->launches = J.per_cycle < 0 ? -1 : 1 + (long long)(J.cycles + 1) + (long long)J.cycles * J.per_cycle;
    for (int r = 0; r < nrhs; ++r) {
      res->iters_max = std::max(res->iters_max, iters[r]);
      res->relres_max = std::max(res->relres_max, relres[r]);
      if (res->iters) res->iters[r] = iters[r];
      if (res->relres) res->relres[r] = relres[r];
    }
  }
  for (int r = 0; r < nrhs; ++r) {
    if (status[r] == -3) st = HELM_ENAN;
    else if (status[r] == 1 && st == HELM_OK) st = HELM_MAXIT;
  }
  if (res) res->status = st;
  if (st == HELM_ENAN) g_err = "non-finite residual in FGMRES";
  return st;
}

template <typename T>
int fgmres_run(helm_ctx* c, int precond, void* net, const double2* b, double2* x, int nrhs, const fgmres_opts& o,
               fgmres_result* res, cudaStream_t caller, const int* maxit_rhs_host = nullptr) {
  FgJob J;
  J.c = c; J.precond = precond; J.net = net; J.b = b; J.x = x; J.nrhs = nrhs; J.o = o;
  J.maxit_rhs_host = maxit_rhs_host; J.caller = caller; J.res = res;
  HTRY(fg_prepare<T>(J));
  for (;;) {
    HTRY(fg_check<T>(J));
    bool done = false;
    HTRY(fg_step<T>(J, &done));
    if (done) break;
  }
  return fg_finish<T>(J);
}

// ===========================================================================
// Block flexible GMRES(m) (the CPU solver of Sec. 4): one block Krylov space for the p
// right-hand sides.  N-length work on the GPU (block Gram matrices, block combinations,
// the operator and the preconditioner on p vectors at once); the small dense algebra in
// FP64 on the host: QR factors of p-vector blocks by Cholesky of their Gram matrix, applied
// twice (CholeskyQR2), block classical Gram-Schmidt applied twice against the basis, and
// the least-squares problem min ||E_1 S - Hbar Y|| by Householder reflections added one
// block column at a time.
// ===========================================================================

// Device buffers of one block solve, released (stream-ordered) on every return path.
struct BlockBufs {
  cudaStream_t s = nullptr;
  std::vector<void*> ptrs;
  void* pinned = nullptr;
  ~BlockBufs() {
    for (void* q : ptrs) cudaFreeAsync(q, s);
    if (pinned) {
      cudaStreamSynchronize(s);
      cudaFreeHost(pinned);
    }
  }
  template <typename P>
  cudaError_t get(P** out, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, bytes, s);
    if (e == cudaSuccess) ptrs.push_back(q);
    *out = (P*)q;
    return e;
  }
};

template <typename T>
int bfgmres_run(helm_ctx* c, int precond, void* net, const double2* b, double2* x, int p, const fgmres_opts& o,
                fgmres_result* res, cudaStream_t caller) {
  typedef typename vec2<T>::type T2;
  const size_t N = level_points(c, 0);
  const int m = o.restart;
  HTRY(ensure_work<T>(c, p, m));
  cudaStream_t s = c->own;
  HCHECK(cudaEventRecord(c->ev_in, caller));
  HCHECK(cudaStreamWaitEvent(s, c->ev_in, 0));
  BlockBufs bb;
  bb.s = s;
  T2 *V, *Z, *Wb;
  double2 *R64, *part, *gram, *dC;
  const int qmax = (m + 1) * p;
  HCHECK(bb.get(&V, (size_t)qmax * N * sizeof(T2)));
  HCHECK(bb.get(&Z, (size_t)m * p * N * sizeof(T2)));
  HCHECK(bb.get(&Wb, (size_t)p * N * sizeof(T2)));
  HCHECK(bb.get(&R64, (size_t)p * N * sizeof(double2)));
  HCHECK(bb.get(&part, (size_t)block_gram_parts(c->nsm) * qmax * p * sizeof(double2)));
  HCHECK(bb.get(&gram, (size_t)qmax * p * sizeof(double2)));
  HCHECK(bb.get(&dC, (size_t)qmax * p * sizeof(double2)));
  if (o.flags & HELM_FLAG_X0_ZERO) HCHECK(cudaMemsetAsync(x, 0, (size_t)p * N * 16, s));
  if (precond == HELM_PREC_JU || precond == HELM_PREC_VU) HTRY(unet_prepare_impl(c, net, p));
  const Op<double> A64 = op_on<double>(c, 0, 0.0);
  const Op<T> AT = op_on<T>(c, 0, 0.0);
  std::vector<double2> hbuf((size_t)qmax * p);
  // coefficient uploads go through a ring of pinned host slots: asynchronous copies, and a
  // slot is rewritten only after a later Gram read has synchronised the stream (at most two
  // uploads happen between two Gram reads)
  constexpr int kRing = 3;
  const size_t slot = (size_t)qmax * p;
  HCHECK(cudaMallocHost(&bb.pinned, kRing * slot * sizeof(double2)));
  double2* ring = (double2*)bb.pinned;
  int ring_i = 0;
  // Gram matrix U^H W (q x p) to the host
  auto gram_host = [&](auto* U, int q, auto* Wv, std::vector<cd>& G) -> int {
    if (block_gram(U, N, q, Wv, N, p, N, part, gram, c->nsm, s) < 0) { g_err = "block Gram: sizes"; return HELM_EINVAL; }
    HLAUNCH();
    HCHECK(cudaMemcpyAsync(hbuf.data(), gram, (size_t)q * p * sizeof(double2), cudaMemcpyDeviceToHost, s));
    HCHECK(cudaStreamSynchronize(s));
    G.resize((size_t)q * p);
    for (size_t i = 0; i < G.size(); ++i) G[i] = cd(hbuf[i].x, hbuf[i].y);
    return HELM_OK;
  };
  // coefficients (q x p, host) to the device (stream-ordered: the previous combine has read
  // dC before this copy lands)
  auto upload = [&](const std::vector<cd>& C, int q) -> int {
    double2* h = ring + (size_t)(ring_i++ % kRing) * slot;
    for (size_t i = 0; i < (size_t)q * p; ++i) h[i] = make_double2(C[i].real(), C[i].imag());
    HCHECK(cudaMemcpyAsync(dC, h, (size_t)q * p * sizeof(double2), cudaMemcpyHostToDevice, s));
    return HELM_OK;
  };
  // blk (p vectors, in place) <- blk R^-1 twice; returns R = R2 R1 (row-major p x p)
  auto qr_block = [&](T2* blk, std::vector<cd>& Rtot) -> int {
    std::vector<cd> G, R1, R1i, R2, R2i;
    HTRY(gram_host(blk, p, blk, G));
    chol_upper(G, p, R1, R1i);
    HTRY(upload(R1i, p));
    if (block_combine(blk, N, p, dC, blk, N, p, N, false, c->nsm, s) < 0) { g_err = "block combine"; return HELM_EINVAL; }
    HLAUNCH();
    HTRY(gram_host(blk, p, blk, G));
    chol_upper(G, p, R2, R2i);
    HTRY(upload(R2i, p));
    if (block_combine(blk, N, p, dC, blk, N, p, N, false, c->nsm, s) < 0) { g_err = "block combine"; return HELM_EINVAL; }
    HLAUNCH();
    Rtot.assign((size_t)p * p, cd(0));
    for (int i = 0; i < p; ++i)
      for (int k = 0; k < p; ++k) {
        cd t = 0;
        for (int l = 0; l < p; ++l) t += R2[(size_t)i * p + l] * R1[(size_t)l * p + k];
        Rtot[(size_t)i * p + k] = t;
      }
    return HELM_OK;
  };
  // right-hand-side norms
  std::vector<cd> G;
  HTRY(gram_host(b, p, b, G));
  std::vector<double> bn(p), rr(p, 0.0);
  for (int k = 0; k < p; ++k) {
    bn[k] = std::sqrt(std::max(0.0, G[(size_t)k * p + k].real()));
    if (bn[k] == 0.0) bn[k] = 1.0;
  }
  std::vector<cd> ident((size_t)p * p, cd(0));
  for (int k = 0; k < p; ++k) ident[(size_t)k * p + k] = 1.0;
  int iters = 0, cycles = 0, st = HELM_OK;
  BlockLS ls;
  for (;;) {
    // true residual in FP64 and its norms
    launch_apply<double>(A64, x, b, R64, p, nullptr, s);
    HLAUNCH();
    HTRY(gram_host(R64, p, R64, G));
    double worst = 0;
    bool finite = true;
    for (int k = 0; k < p; ++k) {
      const double g2 = G[(size_t)k * p + k].real();
      finite = finite && std::isfinite(g2);
      rr[k] = std::sqrt(std::max(0.0, g2)) / bn[k];
      worst = std::max(worst, rr[k]);
    }
    if (!finite) { st = HELM_ENAN; g_err = "non-finite residual in block FGMRES"; break; }
    if (worst <= o.tol) break;
    if (iters >= o.maxit) { st = HELM_MAXIT; break; }
    if (++cycles > o.maxit + 3) { g_err = "block FGMRES cycle guard tripped"; return HELM_ECUDA; }
    // V_1 S = R
    HTRY(upload(ident, p));
    if (block_combine(R64, N, p, dC, V, N, p, N, false, c->nsm, s) < 0) { g_err = "block combine"; return HELM_EINVAL; }
    HLAUNCH();
    std::vector<cd> S;
    HTRY(qr_block(V, S));
    ls.reset(p, m, S);
    int used = 0;
    for (int j = 0; j < m; ++j) {
      T2* Vj = V + (size_t)j * p * N;
      T2* Zj = Z + (size_t)j * p * N;
      HTRY(precond_apply<T>(c, precond, net, Vj, Zj, p, nullptr, s));
      launch_apply<T>(AT, Zj, nullptr, Wb, p, nullptr, s);
      HLAUNCH();
      const int q = (j + 1) * p;
      std::vector<cd> Hc((size_t)q * p, cd(0)), C;
      for (int pass = 0; pass < 2; ++pass) {   // block classical Gram-Schmidt, twice
        HTRY(gram_host(V, q, Wb, C));
        for (size_t i = 0; i < C.size(); ++i) Hc[i] += C[i];
        for (auto& v : C) v = -v;
        HTRY(upload(C, q));
        if (block_combine(V, N, q, dC, Wb, N, p, N, true, c->nsm, s) < 0) { g_err = "block combine"; return HELM_EINVAL; }
        HLAUNCH();
      }
      T2* Vn = V + (size_t)(j + 1) * p * N;
      HTRY(upload(ident, p));
      if (block_combine(Wb, N, p, dC, Vn, N, p, N, false, c->nsm, s) < 0) { g_err = "block combine"; return HELM_EINVAL; }
      HLAUNCH();
      std::vector<cd> Hn;
      HTRY(qr_block(Vn, Hn));
      std::vector<cd> hb((size_t)(j + 2) * p * p, cd(0));
      for (size_t i = 0; i < Hc.size(); ++i) hb[i] = Hc[i];
      for (int i = 0; i < p; ++i)
        for (int k = 0; k < p; ++k) hb[(size_t)(q + i) * p + k] = Hn[(size_t)i * p + k];
      const std::vector<double> est = ls.add(j, hb);
      ++iters;
      used = j + 1;
      bool conv = true;
      for (int k = 0; k < p; ++k) conv = conv && est[k] / bn[k] <= o.tol;
      if (conv || iters >= o.maxit) break;
    }
    // x += [Z_1 .. Z_used] Y
    const std::vector<cd> Y = ls.solve(used);
    HTRY(upload(Y, used * p));
    if (block_combine(Z, N, used * p, dC, x, N, p, N, true, c->nsm, s) < 0) { g_err = "block combine"; return HELM_EINVAL; }
    HLAUNCH();
  }
  HCHECK(cudaStreamSynchronize(s));
  HCHECK(cudaEventRecord(c->ev_out, s));
  HCHECK(cudaStreamWaitEvent(caller, c->ev_out, 0));
  if (res) {
    res->iters_max = iters;
    res->cycles = cycles;
    res->relres_max = 0;
    res->status = st;
    res->launches = -1;   // the preconditioner's launches are not counted here
    for (int k = 0; k < p; ++k) {
      res->relres_max = std::max(res->relres_max, rr[k]);
      if (res->iters) res->iters[k] = iters;
      if (res->relres) res->relres[k] = rr[k];
    }
  }
  return st;
}

int check_common(helm_t h, int nrhs, int dtype) {
  if (!h) { g_err = "null handle"; return HELM_EINVAL; }
  if (nrhs <= 0 || nrhs > 65535) { g_err = "nrhs out of range"; return HELM_EINVAL; }
  if (dtype != HELM_C32 && dtype != HELM_C64) { g_err = "dtype must be HELM_C32 or HELM_C64"; return HELM_EINVAL; }
  if (h->rpp > 0 && nrhs > h->nmedia * h->rpp) {
    g_err = "more right-hand sides than media x right-hand sides per medium";
    return HELM_EINVAL;
  }
  return HELM_OK;
}
int check_level(helm_t h, int level, int need_coarser) {
  if (level < 0 || level + need_coarser >= h->d.levels) { g_err = "level out of range"; return HELM_EINVAL; }
  return HELM_OK;
}

}  // namespace

// ===========================================================================
// bridge used by the U-Net preconditioners (unet.cu)
// ===========================================================================
namespace helm {
int vcycle_public(helm_ctx* c, const void* f, const void* v_in, void* out, int nrhs, int real_bytes, const int* gate,
                  cudaStream_t s) {
  if (real_bytes == 8) { HTRY(ensure_work<double>(c, nrhs, c->d.coarse_its)); return vcycle<double>(c, 0, f, v_in, out, nrhs, gate, s); }
  HTRY(ensure_work<float>(c, nrhs, c->d.coarse_its));
  return vcycle<float>(c, 0, f, v_in, out, nrhs, gate, s);
}
int jacobi_public(helm_ctx* c, int op, const void* f, const void* x_in, void* x_out, int nrhs, int real_bytes,
                  const int* gate, cudaStream_t s) {
  const double beta = op == HELM_OP_M ? c->d.beta : 0.0;
  if (real_bytes == 8) launch_jacobi<double>(op_on<double>(c, 0, beta), c->d.jacobi_w, f, x_in, x_out, nrhs, gate, s);
  else launch_jacobi<float>(op_on<float>(c, 0, beta), (float)c->d.jacobi_w, f, x_in, x_out, nrhs, gate, s);
  HLAUNCH();
  return HELM_OK;
}
int residual_public(helm_ctx* c, int op, const void* b, const void* x, void* r, int nrhs, int real_bytes,
                    const int* gate, cudaStream_t s) {
  const double beta = op == HELM_OP_M ? c->d.beta : 0.0;
  if (real_bytes == 8) launch_apply<double>(op_on<double>(c, 0, beta), x, b, r, nrhs, gate, s);
  else launch_apply<float>(op_on<float>(c, 0, beta), x, b, r, nrhs, gate, s);
  HLAUNCH();
  return HELM_OK;
}
void helm_geometry(helm_ctx* c, int* nx, int* ny, double* h, int* abc_w, double* gmax, const float** k2f,
                   const float** gam) {
  *nx = c->d.nx; *ny = c->d.ny; *h = c->d.h; *abc_w = c->d.abc_width; *gmax = c->d.abc_gamma_max;
  *k2f = c->L[0].k2f;
  *gam = c->gam0;
}
double helm_omega(helm_ctx* c) { return c->d.omega; }
int helm_media(helm_ctx* c, int* rpp) {
  if (rpp) *rpp = c->rpp;
  return c->nmedia;
}
int helm_bc(helm_ctx* c) { return c->d.bc; }
int helm_stencil(helm_ctx* c) { return c->d.stencil; }
void* helm_scratch(helm_ctx* c, int real_bytes, int which, int nrhs) {
  const int r = real_bytes == 8 ? ensure_work<double>(c, nrhs, c->d.coarse_its)
                                : ensure_work<float>(c, nrhs, c->d.coarse_its);
  if (r < 0) return nullptr;
  Work& W = real_bytes == 8 ? c->w64 : c->w32;
  return which == 0 ? W.S0 : W.S1;
}
}  // namespace helm

namespace {
__global__ void k_fill_pattern(float2* __restrict__ v, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long z = (i + 1) * 0x9E3779B97F4A7C15ull;
    v[i] = make_float2((float)((z >> 40) & 0xFFFF) / 65536.f - 0.5f, (float)((z >> 20) & 0xFFFF) / 65536.f - 0.5f);
  }
}
__global__ void k_sub_inplace(double2* __restrict__ e, const double2* __restrict__ xt, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double2 a = e[i], b = xt[i];
    e[i] = make_double2(a.x - b.x, a.y - b.y);
  }
}
uint64_t host_splitmix(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* helm_last_error(void) { return g_err.c_str(); }

int helm_desc_default(helm_desc* d, int nx, int ny) {
  if (!d) { g_err = "null desc"; return HELM_EINVAL; }
  std::memset(d, 0, sizeof(*d));
  d->nx = nx; d->ny = ny;
  d->h = 1.0 / (double)nx;
  d->omega = 2.0 * 3.14159265358979323846 / 10.0 / d->h;
  d->beta = 0.5;
  d->abc_width = 16;
  d->abc_gamma_max = 1.0;
  d->levels = 3;
  d->nu1 = 1; d->nu2 = 1;
  d->jacobi_w = 0.8;
  d->coarse_its = 10;
  return HELM_OK;
}

int helm_setup(const helm_desc* desc, const float* kappa2, helm_stream_t stream, helm_t* out) {
  return helm_setup_media(desc, kappa2, 1, 0, stream, out);
}

int helm_setup_media(const helm_desc* desc, const float* kappa2, int nmedia, int rpp, helm_stream_t stream,
                     helm_t* out) {
  if (!desc || !kappa2 || !out) { g_err = "null argument"; return HELM_EINVAL; }
  if (nmedia < 1 || rpp < 0 || (nmedia > 1 && rpp < 1)) {
    g_err = "nmedia must be >= 1, and rpp >= 1 when there is more than one medium";
    return HELM_EINVAL;
  }
  const helm_desc& d = *desc;
  if (d.levels < 1 || d.levels > 12) { g_err = "levels must be in 1..12"; return HELM_EINVAL; }
  const int div = 1 << (d.levels - 1);
  if (d.nx <= 0 || d.ny <= 0 || d.nx % div || d.ny % div) {
    g_err = "nx, ny must be positive multiples of 2^(levels-1)";
    return HELM_EINVAL;
  }
  if (d.coarse_its < 1 || d.coarse_its > 32) { g_err = "coarse_its must be in 1..32"; return HELM_EINVAL; }
  if (d.nu1 < 0 || d.nu2 < 0 || d.h <= 0 || d.abc_width < 0) { g_err = "bad smoothing/mesh/layer parameter"; return HELM_EINVAL; }
  if (d.bc < HELM_BC_DIRICHLET || d.bc > HELM_BC_REPLICATE) { g_err = "bc must be a HELM_BC_* value"; return HELM_EINVAL; }
  if (d.stencil != HELM_STENCIL_5PT && d.stencil != HELM_STENCIL_COMPACT4) {
    g_err = "stencil must be a HELM_STENCIL_* value";
    return HELM_EINVAL;
  }
  if (d.stencil == HELM_STENCIL_COMPACT4 && d.bc != HELM_BC_DIRICHLET) {
    g_err = "the compact fourth-order stencil is built for Dirichlet boundaries only";
    return HELM_EUNSUPPORTED;
  }
  if (d.bc == HELM_BC_REFLECT && ((d.nx >> (d.levels - 1)) < 2 || (d.ny >> (d.levels - 1)) < 2)) {
    g_err = "reflection boundaries need the coarsest level at least 2 x 2";
    return HELM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  helm_ctx* c = new helm_ctx();
  c->d = d;
  c->fused_coarse = !(d.flags & HELM_DESC_MULTIKERNEL_COARSE);
  c->cluster_coarse = !(d.flags & (HELM_DESC_MULTIKERNEL_COARSE | HELM_DESC_SINGLE_CTA_COARSE));
  HCHECK(cudaGetDevice(&c->device));
  HCHECK(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device));
  c->nmedia = nmedia;
  c->rpp = nmedia > 1 ? rpp : 0;
  size_t total = 0;
  for (int l = 0; l < d.levels; ++l) total += (size_t)nmedia * (d.nx >> l) * (d.ny >> l) * 12 + 512;
  if (cudaMalloc(&c->level_mem, total) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    g_err = "level allocation failed";
    return HELM_ENOMEM;
  }
  Arena a{(char*)c->level_mem, total, 0};
  for (int l = 0; l < d.levels; ++l) {
    Level L;
    L.nx = d.nx >> l; L.ny = d.ny >> l;
    L.h = d.h * (double)(1 << l);
    L.abc_w = d.abc_width >> l;
    L.bc = d.bc;
    L.order = d.stencil == HELM_STENCIL_COMPACT4 ? 4 : 2;
    L.rpp = c->rpp;
    size_t n = (size_t)nmedia * L.nx * L.ny;
    L.k2f = (float*)a.take(n * 4);
    L.k2d = (double*)a.take(n * 8);
    c->L.push_back(L);
  }
  const size_t n0 = (size_t)d.nx * d.ny;
  HCHECK(cudaMemcpyAsync(c->L[0].k2f, kappa2, (size_t)nmedia * n0 * 4, cudaMemcpyDeviceToDevice, s));
  launch_widen_kappa2(c->L[0].k2f, c->L[0].k2d, (size_t)nmedia * n0, s);
  for (int l = 1; l < d.levels; ++l) {
    const size_t nf = (size_t)c->L[l - 1].nx * c->L[l - 1].ny, nc = (size_t)c->L[l].nx * c->L[l].ny;
    for (int q = 0; q < nmedia; ++q)
      launch_coarsen_kappa2(c->L[l - 1].k2d + q * nf, c->L[l - 1].nx, c->L[l - 1].ny, c->L[l].k2d + q * nc,
                            c->L[l].k2f + q * nc, s);
  }
  HLAUNCH();
  HCHECK(cudaMalloc(&c->gam0, n0 * 4));
  gamma_field(d.ny, d.nx, d.abc_width, (float)d.abc_gamma_max, c->gam0, s);
  HLAUNCH();
  HCHECK(cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking));
  HCHECK(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
  HCHECK(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
  HCHECK(cudaStreamSynchronize(s));
  *out = c;
  return HELM_OK;
}

void helm_destroy(helm_t h) {
  if (!h) return;
  cudaDeviceSynchronize();
  drop_graphs(h);
  unet_release_ctx(h);
  free_work(h->w32);
  free_work(h->w64);
  if (h->level_mem) cudaFree(h->level_mem);
  if (h->gam0) cudaFree(h->gam0);
  if (h->h_done) cudaFreeHost(h->h_done);
  if (h->own) cudaStreamDestroy(h->own);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  delete h;
}

int helm_level_shape(helm_t h, int level, int* nx, int* ny) {
  if (!h) { g_err = "null handle"; return HELM_EINVAL; }
  HTRY(check_level(h, level, 0));
  if (nx) *nx = h->L[level].nx;
  if (ny) *ny = h->L[level].ny;
  return HELM_OK;
}

int helm_level_kappa2(helm_t h, int level, double* out) {
  if (!h || !out) { g_err = "null argument"; return HELM_EINVAL; }
  HTRY(check_level(h, level, 0));
  HCHECK(cudaMemcpy(out, h->L[level].k2d, level_points(h, level) * 8, cudaMemcpyDeviceToDevice));
  return HELM_OK;
}

int helm_apply(helm_t h, int op, int level, const void* x, void* y, int nrhs, int dtype, helm_stream_t stream) {
  if (op != HELM_OP_RHS) return helm_residual(h, op, level, nullptr, x, y, nrhs, dtype, stream);
  HTRY(check_common(h, nrhs, dtype));
  HTRY(check_level(h, level, 0));
  if (!x || !y || x == y) { g_err = "bad vectors (y must not alias x)"; return HELM_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)nrhs * level_points(h, level) * (dtype == HELM_C32 ? 8 : 16);
  if (h->d.stencil != HELM_STENCIL_COMPACT4) HCHECK(cudaMemcpyAsync(y, x, bytes, cudaMemcpyDeviceToDevice, s));
  else if (dtype == HELM_C32) launch_rhs_weight<float>(op_on<float>(h, level, 0.0), x, y, nrhs, s);
  else launch_rhs_weight<double>(op_on<double>(h, level, 0.0), x, y, nrhs, s);
  HLAUNCH();
  return HELM_OK;
}

int helm_residual(helm_t h, int op, int level, const void* b, const void* x, void* r, int nrhs, int dtype,
                  helm_stream_t stream) {
  HTRY(check_common(h, nrhs, dtype));
  HTRY(check_level(h, level, 0));
  if (op != HELM_OP_A && op != HELM_OP_M) { g_err = "op must be HELM_OP_A or HELM_OP_M"; return HELM_EINVAL; }
  if (!x || !r) { g_err = "null vector"; return HELM_EINVAL; }
  if (r == x || r == b) { g_err = "the output must not alias an input"; return HELM_EINVAL; }
  const double beta = (op == HELM_OP_M) ? h->d.beta : 0.0;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == HELM_C32) launch_apply<float>(op_on<float>(h, level, beta), x, b, r, nrhs, nullptr, s);
  else launch_apply<double>(op_on<double>(h, level, beta), x, b, r, nrhs, nullptr, s);
  HLAUNCH();
  return HELM_OK;
}

int helm_jacobi(helm_t h, int op, int level, const void* b, const void* x_in, void* x_out, int nrhs, int dtype,
                helm_stream_t stream) {
  HTRY(check_common(h, nrhs, dtype));
  HTRY(check_level(h, level, 0));
  if (op != HELM_OP_A && op != HELM_OP_M) { g_err = "op must be HELM_OP_A or HELM_OP_M"; return HELM_EINVAL; }
  if (!b || !x_out || x_in == x_out) { g_err = "bad vectors (x_out must not alias x_in)"; return HELM_EINVAL; }
  const double beta = (op == HELM_OP_M) ? h->d.beta : 0.0;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == HELM_C32)
    launch_jacobi<float>(op_on<float>(h, level, beta), (float)h->d.jacobi_w, b, x_in, x_out, nrhs, nullptr, s);
  else
    launch_jacobi<double>(op_on<double>(h, level, beta), h->d.jacobi_w, b, x_in, x_out, nrhs, nullptr, s);
  HLAUNCH();
  return HELM_OK;
}

int helm_restrict(helm_t h, int level, const void* fine, void* coarse, int nrhs, int dtype, helm_stream_t stream) {
  HTRY(check_common(h, nrhs, dtype));
  HTRY(check_level(h, level, 1));
  if (!fine || !coarse) { g_err = "null vector"; return HELM_EINVAL; }
  const Level& L = h->L[level];
  if (dtype == HELM_C32) launch_restrict<float>(L.nx, L.ny, fine, coarse, nrhs, nullptr, (cudaStream_t)stream);
  else launch_restrict<double>(L.nx, L.ny, fine, coarse, nrhs, nullptr, (cudaStream_t)stream);
  HLAUNCH();
  return HELM_OK;
}

int helm_prolong_add(helm_t h, int level, const void* coarse, void* fine, int nrhs, int dtype,
                     helm_stream_t stream) {
  HTRY(check_common(h, nrhs, dtype));
  HTRY(check_level(h, level, 1));
  if (!fine || !coarse) { g_err = "null vector"; return HELM_EINVAL; }
  const Level& L = h->L[level];
  const Level& C = h->L[level + 1];
  if (dtype == HELM_C32) launch_prolong_add<float>(C.nx, C.ny, L.nx, L.ny, coarse, fine, nrhs, nullptr, (cudaStream_t)stream);
  else launch_prolong_add<double>(C.nx, C.ny, L.nx, L.ny, coarse, fine, nrhs, nullptr, (cudaStream_t)stream);
  HLAUNCH();
  return HELM_OK;
}

int helm_coarse_solve(helm_t h, const void* f, void* x, int nrhs, int dtype, helm_stream_t stream) {
  HTRY(check_common(h, nrhs, dtype));
  if (!f || !x || f == x) { g_err = "bad vectors"; return HELM_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == HELM_C32) {
    HTRY(ensure_work<float>(h, nrhs, h->d.coarse_its));
    return coarse_gmres<float>(h, f, x, nrhs, nullptr, s);
  }
  HTRY(ensure_work<double>(h, nrhs, h->d.coarse_its));
  return coarse_gmres<double>(h, f, x, nrhs, nullptr, s);
}

int sl_vcycle(helm_t h, const void* f, void* x, int nrhs, int dtype, int x_is_zero, helm_stream_t stream) {
  HTRY(check_common(h, nrhs, dtype));
  if (!f || !x || f == x) { g_err = "bad vectors (f and x must differ)"; return HELM_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == HELM_C32) {
    HTRY(ensure_work<float>(h, nrhs, h->d.coarse_its));
    return vcycle<float>(h, 0, f, x_is_zero ? nullptr : x, x, nrhs, nullptr, s);
  }
  HTRY(ensure_work<double>(h, nrhs, h->d.coarse_its));
  return vcycle<double>(h, 0, f, x_is_zero ? nullptr : x, x, nrhs, nullptr, s);
}

int fgmres_solve(helm_t h, int precond, void* net, const void* b, void* x, int nrhs, const fgmres_opts* opts,
                 fgmres_result* result, helm_stream_t stream) {
  HTRY(check_common(h, nrhs, HELM_C32));
  if (!b || !x || !opts) { g_err = "null argument"; return HELM_EINVAL; }
  fgmres_opts o = *opts;
  if (o.restart < 1 || o.restart > 32) { g_err = "restart must be in 1..32"; return HELM_EINVAL; }
  if (!(o.tol >= 0) || o.maxit < 0) { g_err = "bad tol/maxit"; return HELM_EINVAL; }
  if ((precond == HELM_PREC_JU || precond == HELM_PREC_VU) && !net) { g_err = "U-Net preconditioner needs net"; return HELM_EINVAL; }
  cudaStream_t caller = (cudaStream_t)stream;
  const size_t bytes = (size_t)nrhs * h->d.nx * h->d.ny * 16;
  const bool fp64 = (o.flags & HELM_FLAG_FP64) != 0;
  const void* bd = b;
  void* xd = x;
  if (o.flags & HELM_FLAG_HOST_IO) {
    if (fp64) HTRY(ensure_work<double>(h, nrhs, o.restart));
    else HTRY(ensure_work<float>(h, nrhs, o.restart));
    Work& W = fp64 ? h->w64 : h->w32;
    HCHECK(cudaMemcpyAsync(W.bx, b, bytes, cudaMemcpyHostToDevice, caller));
    if (!(o.flags & HELM_FLAG_X0_ZERO)) HCHECK(cudaMemcpyAsync(W.xx, x, bytes, cudaMemcpyHostToDevice, caller));
    bd = W.bx;
    xd = W.xx;
  }
  auto run = [&](int pc, void* nt, const fgmres_opts& oo, fgmres_result* rs) {
    return fp64 ? fgmres_run<double>(h, pc, nt, (const double2*)bd, (double2*)xd, nrhs, oo, rs, caller)
                : fgmres_run<float>(h, pc, nt, (const double2*)bd, (double2*)xd, nrhs, oo, rs, caller);
  };
  const bool fallback =
      (o.flags & HELM_FLAG_FALLBACK_V) && (precond == HELM_PREC_JU || precond == HELM_PREC_VU);
  int r;
  if (!fallback) {
    r = run(precond, net, o, result);
    if (result) result->fallbacks = 0;
  } else {
    // U-Net solve first; right-hand sides left above tol are solved again with M_V from
    // their iterate (zeroed where it is not finite), the others finish at the first check
    std::vector<int> it1(nrhs), it2(nrhs);
    std::vector<double> rr1(nrhs), rr2(nrhs);
    fgmres_result r1{}, r2{};
    r1.iters = it1.data(); r1.relres = rr1.data();
    r2.iters = it2.data(); r2.relres = rr2.data();
    r = run(precond, net, o, &r1);
    if (r < 0 && r != HELM_ENAN) return r;
    const size_t N = (size_t)h->d.nx * h->d.ny;
    int nfail = 0;
    for (int k = 0; k < nrhs; ++k) {
      if (rr1[k] <= o.tol) continue;
      ++nfail;
      if (!std::isfinite(rr1[k])) HCHECK(cudaMemsetAsync((double2*)xd + (size_t)k * N, 0, N * 16, caller));
    }
    fgmres_result fin = r1;
    if (nfail) {
      fgmres_opts o2 = o;
      o2.flags &= ~(HELM_FLAG_X0_ZERO | HELM_FLAG_HOST_IO | HELM_FLAG_FALLBACK_V);
      r = run(HELM_PREC_V, nullptr, o2, &r2);
      if (r < 0 && r != HELM_ENAN) return r;
      fin = r2;
      fin.cycles = r1.cycles + r2.cycles;
      fin.launches = (r1.launches < 0 || r2.launches < 0) ? -1 : r1.launches + r2.launches;
      fin.iters_max = 0;
      for (int k = 0; k < nrhs; ++k) {
        it2[k] += it1[k];
        fin.iters_max = std::max(fin.iters_max, it2[k]);
      }
    }
    if (result) {
      const std::vector<int>& it = nfail ? it2 : it1;
      const std::vector<double>& rr = nfail ? rr2 : rr1;
      for (int k = 0; k < nrhs; ++k) {
        if (result->iters) result->iters[k] = it[k];
        if (result->relres) result->relres[k] = rr[k];
      }
      result->iters_max = fin.iters_max;
      result->cycles = fin.cycles;
      result->relres_max = fin.relres_max;
      result->status = fin.status;
      result->launches = fin.launches;
      result->fallbacks = nfail;
    }
  }
  if (r < 0 && r != HELM_ENAN) return r;
  if (o.flags & HELM_FLAG_HOST_IO) {
    HCHECK(cudaMemcpyAsync(x, xd, bytes, cudaMemcpyDeviceToHost, caller));
    HCHECK(cudaStreamSynchronize(caller));
  }
  return r;
}

int fgmres_solve_batch(int nh, helm_t* hs, int precond, void* const* nets, const void* const* b, void* const* x,
                       const int* nrhs, const fgmres_opts* opts, fgmres_result* results, helm_stream_t stream) {
  if (nh < 1 || !hs || !b || !x || !nrhs || !opts) { g_err = "fgmres_solve_batch: null argument"; return HELM_EINVAL; }
  const fgmres_opts o = *opts;
  if (o.restart < 1 || o.restart > 32) { g_err = "restart must be in 1..32"; return HELM_EINVAL; }
  if (!(o.tol >= 0) || o.maxit < 0) { g_err = "bad tol/maxit"; return HELM_EINVAL; }
  if (o.flags & (HELM_FLAG_HOST_IO | HELM_FLAG_FP64 | HELM_FLAG_FALLBACK_V | HELM_FLAG_NO_GRAPH)) {
    g_err = "fgmres_solve_batch takes device vectors and captured FP32 cycles (no HOST_IO, FP64, FALLBACK_V, NO_GRAPH)";
    return HELM_EUNSUPPORTED;
  }
  const bool unet = precond == HELM_PREC_JU || precond == HELM_PREC_VU;
  std::vector<FgJob> jobs(nh);
  for (int i = 0; i < nh; ++i) {
    HTRY(check_common(hs[i], nrhs[i], HELM_C32));
    if (!b[i] || !x[i]) { g_err = "fgmres_solve_batch: null vector"; return HELM_EINVAL; }
    for (int k = 0; k < i; ++k) {
      if (hs[k] == hs[i]) { g_err = "fgmres_solve_batch: a handle appears twice"; return HELM_EINVAL; }
      // a network keeps one activation workspace, sized for one grid
      if (unet && nets && nets[k] == nets[i] &&
          (hs[k]->d.nx != hs[i]->d.nx || hs[k]->d.ny != hs[i]->d.ny)) {
        g_err = "fgmres_solve_batch: handles of different grids need their own network handles";
        return HELM_EINVAL;
      }
    }
    if (unet && (!nets || !nets[i])) { g_err = "U-Net preconditioner needs a network per handle"; return HELM_EINVAL; }
    FgJob& J = jobs[i];
    J.c = hs[i]; J.precond = precond; J.net = unet ? nets[i] : nullptr; J.b = (const double2*)b[i];
    J.x = (double2*)x[i]; J.nrhs = nrhs[i]; J.o = o; J.caller = (cudaStream_t)stream;
    J.res = results ? &results[i] : nullptr;
  }
  for (auto& J : jobs) HTRY(fg_prepare<float>(J));
  // rounds: every unfinished handle's residual check is enqueued on its stream, then each
  // in turn is waited for and given its next cycle, so the handles' cycles overlap
  for (int left = nh; left > 0;) {
    for (auto& J : jobs)
      if (!J.finished) HTRY(fg_check<float>(J));
    for (auto& J : jobs) {
      if (J.finished) continue;
      bool done = false;
      HTRY(fg_step<float>(J, &done));
      if (done) { J.finished = true; --left; }
    }
  }
  int worst = HELM_OK;
  for (auto& J : jobs) {
    const int r = fg_finish<float>(J);
    if (r < 0 && worst >= 0) worst = r;
    else if (r == HELM_MAXIT && worst == HELM_OK) worst = r;
  }
  return worst;
}

int bfgmres_solve(helm_t h, int precond, void* net, const void* b, void* x, int nrhs, const fgmres_opts* opts,
                  fgmres_result* result, helm_stream_t stream) {
  HTRY(check_common(h, nrhs, HELM_C32));
  if (!b || !x || !opts) { g_err = "null argument"; return HELM_EINVAL; }
  fgmres_opts o = *opts;
  if (nrhs > 16) { g_err = "block size (nrhs) must be at most 16"; return HELM_EINVAL; }
  if (h->nmedia > 1) { g_err = "block FGMRES needs one operator for every column (one medium)"; return HELM_EUNSUPPORTED; }
  if (o.flags & HELM_FLAG_FALLBACK_V) { g_err = "HELM_FLAG_FALLBACK_V is for fgmres_solve"; return HELM_EUNSUPPORTED; }
  if (o.restart < 1 || o.restart > 32 || (o.restart + 1) * nrhs * nrhs > 4608) {
    g_err = "restart must be in 1..32 with (restart + 1) nrhs^2 <= 4608";
    return HELM_EINVAL;
  }
  if (!(o.tol >= 0) || o.maxit < 0) { g_err = "bad tol/maxit"; return HELM_EINVAL; }
  if ((precond == HELM_PREC_JU || precond == HELM_PREC_VU) && !net) { g_err = "U-Net preconditioner needs net"; return HELM_EINVAL; }
  cudaStream_t caller = (cudaStream_t)stream;
  const size_t bytes = (size_t)nrhs * h->d.nx * h->d.ny * 16;
  const bool fp64 = (o.flags & HELM_FLAG_FP64) != 0;
  const void* bd = b;
  void* xd = x;
  if (o.flags & HELM_FLAG_HOST_IO) {
    if (fp64) HTRY(ensure_work<double>(h, nrhs, o.restart));
    else HTRY(ensure_work<float>(h, nrhs, o.restart));
    Work& W = fp64 ? h->w64 : h->w32;
    HCHECK(cudaMemcpyAsync(W.bx, b, bytes, cudaMemcpyHostToDevice, caller));
    if (!(o.flags & HELM_FLAG_X0_ZERO)) HCHECK(cudaMemcpyAsync(W.xx, x, bytes, cudaMemcpyHostToDevice, caller));
    bd = W.bx;
    xd = W.xx;
  }
  if (result) result->fallbacks = 0;
  int r = fp64 ? bfgmres_run<double>(h, precond, net, (const double2*)bd, (double2*)xd, nrhs, o, result, caller)
               : bfgmres_run<float>(h, precond, net, (const double2*)bd, (double2*)xd, nrhs, o, result, caller);
  if (r < 0 && r != HELM_ENAN) return r;
  if (o.flags & HELM_FLAG_HOST_IO) {
    HCHECK(cudaMemcpyAsync(x, xd, bytes, cudaMemcpyDeviceToHost, caller));
    HCHECK(cudaStreamSynchronize(caller));
  }
  return r;
}

int helm_gen_pairs(helm_t h, int count, unsigned long long seed, int kmax, void* r, void* e, helm_stream_t stream) {
  HTRY(check_common(h, count, HELM_C64));
  if (!r || !e || r == e || kmax < 1 || kmax > 1000) { g_err = "bad arguments"; return HELM_EINVAL; }
  if (h->nmedia > 1) { g_err = "training pairs are generated on a handle of one medium"; return HELM_EUNSUPPORTED; }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = (size_t)h->d.nx * h->d.ny;
  HTRY(ensure_work<float>(h, count, h->d.coarse_its > 10 ? h->d.coarse_its : 10));
  Work& W = h->w32;
  // x ~ CN(0,1) into e; b = A x into r (FP64)
  complex_normal(seed, count, N, (double2*)e, s);
  launch_apply<double>(op_on<double>(h, 0, 0.0), e, nullptr, r, count, nullptr, s);
  HLAUNCH();
  // k_j = 1 + floor(U_j kmax), U_j the j-th uniform of stream `seed`
  std::vector<int> ks(count);
  for (int j = 0; j < count; ++j) {
    double u = ((double)(host_splitmix(seed, (uint64_t)j) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    ks[j] = 1 + (int)std::floor(u * kmax);
    if (ks[j] > kmax) ks[j] = kmax;
  }
  // x~ = k_j FGMRES(M_V) iterations from 0 (Eq. 3.8)
  fgmres_opts o{std::max(10, kmax), 0.0, kmax, HELM_FLAG_X0_ZERO};
  if (o.restart > 32) o.restart = 32;
  fgmres_result res{};
  int st = fgmres_run<float>(h, HELM_PREC_V, nullptr, (const double2*)r, W.xx, count, o, &res, s, ks.data());
  if (st < 0) return st;
  // r = b - A x~ ; e = x - x~ (Eq. 3.9)
  launch_apply<double>(op_on<double>(h, 0, 0.0), W.xx, r, r, count, nullptr, s);
  k_sub_inplace<<<1024, 256, 0, s>>>((double2*)e, W.xx, (size_t)count * N);
  HLAUNCH();
  return HELM_OK;
}

int helm_tile_choice(helm_t h, int kernel, int level, int nrhs, int* seg) {
  if (!h || !seg || (kernel != 0 && kernel != 1) || level < 0 || level + 1 >= h->d.levels || nrhs < 1) {
    g_err = "helm_tile_choice: bad arguments";
    return HELM_EINVAL;
  }
  auto it = h->seg.find(std::make_tuple(kernel, level, nrhs));
  *seg = it == h->seg.end() ? 0 : it->second;
  return HELM_OK;
}

int helm_set_tile_choice(helm_t h, int kernel, int level, int nrhs, int seg) {
  if (!h || (kernel != 0 && kernel != 1) || level < 0 || level + 1 >= h->d.levels || nrhs < 1 ||
      !(seg == -1 || seg == 0 || seg == 4 || seg == 8 || seg == 16 || seg == 32)) {
    g_err = "helm_set_tile_choice: bad arguments";
    return HELM_EINVAL;
  }
  const auto key = std::make_tuple(kernel, level, nrhs);
  if (seg == 0) h->seg.erase(key);
  else h->seg[key] = seg;
  drop_graphs(h);   // captured cycles baked in the previous choice
  return HELM_OK;
}

int helm_time_kernel(helm_t h, int kernel, int nrhs, int reps, helm_stream_t stream, float* ms, double* bytes) {
  HTRY(check_common(h, nrhs, HELM_C32));
  if (reps < 1 || !ms || !bytes) { g_err = "bad reps/outputs"; return HELM_EINVAL; }
  HTRY(ensure_work<float>(h, nrhs, 10));
  Work& W = h->w32;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = level_points(h, 0), Nc1 = level_points(h, std::min(1, h->d.levels - 1));
  const size_t es = 8, vstride = (size_t)nrhs * N;
  char* V = (char*)W.V;
  const Op<float> A = op_on<float>(h, 0, 0.0), M = op_on<float>(h, 0, h->d.beta);
  const int nb = vec_blocks(N, nrhs, h->nsm);
  // active flags on, finite Hessenberg entries
  HCHECK(cudaMemsetAsync(W.fst.H, 0, (size_t)nrhs * (W.fst.m + 1) * W.fst.m * 16, s));
  k_fill_pattern<<<1024, 256, 0, s>>>((float2*)V, (size_t)nrhs * N);   // nonzero data in v_0
  {  // a nonzero right-hand side on the coarsest level so its solve does real work
    const int lc = h->d.levels - 1;
    HCHECK(cudaMemcpyAsync(W.F[lc], V, (size_t)nrhs * level_points(h, lc) * es, cudaMemcpyDeviceToDevice, s));
  }
  std::vector<int> ones(nrhs, 1), many(nrhs, 1 << 30);
  HCHECK(cudaMemcpyAsync(W.fst.active, ones.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));
  // a step limit never reached and a zero tolerance keep every right-hand side active
  HCHECK(cudaMemcpyAsync(W.fst.kmax, many.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));
  HCHECK(cudaMemsetAsync(W.fst.tol_abs, 0, (size_t)nrhs * sizeof(double), s));
  HCHECK(cudaMemsetAsync(W.fst.proj, 0, (size_t)nrhs * kProjMax * sizeof(double2), s));
  HCHECK(cudaStreamSynchronize(s));
  auto run = [&](void) -> int {
    switch (kernel) {
      case 0: launch_apply<float>(A, V, nullptr, V + vstride * es, nrhs, nullptr, s); break;
      case 1: launch_resid_restrict<float>(M, 0.8f, V, nullptr, W.F[1], nrhs, nullptr, s); break;
      case 2: launch_prolong_jacobi<float>(M, 0.8f, V, nullptr, true, W.E[1], h->L[1].nx, h->L[1].ny,
                                           V + vstride * es, nrhs, nullptr, s); break;
      case 3: launch_arnoldi_sweep<float>(1, A, nullptr, V, vstride, nrhs, W.fst, 4, nb, s); break;
      case 6: launch_arnoldi_sweep<float>(0, A, V + 6 * vstride * es, V, vstride, nrhs, W.fst, 4, nb, s); break;
      case 4: return vcycle<float>(h, 0, V, nullptr, V + vstride * es, nrhs, nullptr, s);
      case 5: return coarse_gmres<float>(h, W.F[h->d.levels - 1], W.E[h->d.levels - 1], nrhs, nullptr, s);
      default: g_err = "unknown kernel id"; return HELM_EINVAL;
    }
    return HELM_OK;
  };
  const double n = (double)N * nrhs, nc = (double)Nc1 * nrhs;
  switch (kernel) {
    case 0: *bytes = 20.0 * n; break;
    case 1: *bytes = 12.0 * n + 8.0 * nc; break;
    case 2: *bytes = 20.0 * n + 8.0 * nc; break;
    case 3: *bytes = 56.0 * n; break;   // w and v_0..v_4 read, w written
    case 6: *bytes = 60.0 * n; break;   // z, kappa^2 and v_0..v_4 read, w written
    default: *bytes = 0.0; break;
  }
  HTRY(run());  // warm-up
  cudaEvent_t e0, e1;
  HCHECK(cudaEventCreate(&e0));
  HCHECK(cudaEventCreate(&e1));
  HCHECK(cudaEventRecord(e0, s));
  for (int r = 0; r < reps; ++r) HTRY(run());
  HCHECK(cudaEventRecord(e1, s));
  HCHECK(cudaEventSynchronize(e1));
  float t = 0;
  HCHECK(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t / reps;
  HLAUNCH();
  return HELM_OK;
}

}  // extern "C"
