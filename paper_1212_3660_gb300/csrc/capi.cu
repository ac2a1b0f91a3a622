// Host engine and C ABI of the flexible shifted-Krylov solver.
//
// fks_solve runs Algorithm 3 (flexible Arnoldi) for every source in lockstep
// and Algorithm 4 (per-shift FGMRES / FFOM) after every step, with the inner
// preconditioner solves (Section 4) done by multigrid cycles and a defect
// correction in complex128. All per-step state lives in device memory; the
// host only enqueues kernels and reads small flags to decide when a loop ends.
#include <algorithm>
#include <atomic>
#include <limits>
#include <complex>
#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <thread>
#include <memory>
#include <deque>
#include <condition_variable>
#include <chrono>
#include <string>
#include <vector>

#include "../../include/fks.h"
#include "common.cuh"
#include "grid.cuh"
#include "krylov.cuh"
#include "csr.cuh"
#include "assemble_tc.cuh"
#include "cluster.cuh"
#include "coop.cuh"
#include "sensitivity.cuh"
#include "monitors.cuh"
#include "amg.cuh"

namespace fks {

static thread_local std::string g_err;
// Graph capture/instantiation and kernel attribute changes are serialised
// across threads (the server builds graphs from several worker threads).
static std::mutex g_build_mu;
// Serialises the host-side CUDA calls of concurrent server batches.
void set_error(const std::string& msg) { g_err = msg; }
const char* get_error() { return g_err.c_str(); }

constexpr int NU1 = 2;  // pre-smoothing red-black sweeps
constexpr int NU2 = 2;  // post-smoothing sweeps
constexpr double BREAKDOWN_RTOL = 1e-13;

struct CudaError {
  cudaError_t e;
  const char* where;
};

// Test hook (fks_debug_fail_allocs): the next this-many workspace reservations
// fail as cudaMalloc would when the device is out of memory.
static std::atomic<int> g_fail_allocs{0};

#define CK(x)                                            \
  do {                                                   \
    cudaError_t e_ = (x);                                \
    if (e_ != cudaSuccess) throw CudaError{e_, #x};      \
  } while (0)

// One growable device buffer carved into aligned pieces.
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  cudaStream_t astream = nullptr;  // stream-ordered allocation on this stream when set
  void reserve(size_t bytes) {
    if (bytes <= cap) return;
    if (g_fail_allocs.load() > 0 && g_fail_allocs.fetch_sub(1) > 0)
      throw CudaError{cudaErrorMemoryAllocation, "cudaMalloc(workspace) (injected failure)"};
    if (base) {
      if (astream) cudaFreeAsync(base, astream); else cudaFree(base);
    }
    base = nullptr;
    cap = 0;
    cudaError_t e = astream ? cudaMallocAsync((void**)&base, bytes, astream) : cudaMalloc(&base, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw CudaError{e, "cudaMalloc(workspace)"};
    }
    cap = bytes;
  }
  void release() {
    if (base) {
      if (astream) cudaFreeAsync(base, astream); else cudaFree(base);
    }
    base = nullptr;
    cap = 0;
  }
  void reset() { off = 0; }
  template <typename T>
  T* take(size_t count) {
    size_t bytes = ((count * sizeof(T)) + 255) & ~(size_t)255;
    T* p = (T*)(base ? base + off : nullptr);
    off += bytes;
    return p;
  }
};

// Event timing of one selected kernel class plus a count of all launches.
struct Prof {
  int cls = -1, level = -1;
  std::vector<cudaEvent_t> ev;
  std::vector<double> bytes, flops;
  size_t used = 0;
  int64_t launches = 0, all_launches = 0;
  double ms = 0.0, tot_bytes = 0.0, tot_flops = 0.0;
  bool open = false;
  bool match(int c, int l) const { return cls >= 0 && c == cls && (level < 0 || l == level); }
  void begin(int c, int l, double b, double f, cudaStream_t s) {
    ++all_launches;
    open = match(c, l);
    if (!open) return;
    if (2 * used + 2 > ev.size()) {
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      ev.push_back(e0);
      ev.push_back(e1);
      bytes.push_back(0);
      flops.push_back(0);
    }
    cudaEventRecord(ev[2 * used], s);
    bytes[used] = b;
    flops[used] = f;
  }
  void end(cudaStream_t s) {
    if (!open) return;
    cudaEventRecord(ev[2 * used + 1], s);
    ++used;
    open = false;
  }
  void collect() {
    for (size_t i = 0; i < used; ++i) {
      cudaEventSynchronize(ev[2 * i + 1]);
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]);
      ms += t;
      tot_bytes += bytes[i];
      tot_flops += flops[i];
      ++launches;
    }
    used = 0;
  }
  void release() {
    for (auto e : ev) cudaEventDestroy(e);
    ev.clear();
  }
};

// Everything one in-flight solve owns: workspace, the captured step-loop
// graph, instrumentation. fks_solve uses the operator's own lane; the server
// gives each concurrent batch a lane of its own.
struct Lane {
  Arena ws;
  Arena tcws;  // slices of the tensor-core assembly
  Arena xws;   // server lanes: one source's x_j, assembled there and delivered
  Prof prof;
  cudaGraphExec_t graph = nullptr;
  std::vector<double> graph_key;
  int graph_outer = 0, graph_inner = 0;
  // a second stream that copies x_j to host memory while the true residuals run
  cudaStream_t side = nullptr;
  cudaEvent_t ev_x = nullptr, ev_copied = nullptr;
  void side_init() {
    if (side) return;
    CK(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ev_x, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_copied, cudaEventDisableTiming));
  }
  void release() {
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
    if (side) {
      cudaStreamSynchronize(side);
      cudaStreamDestroy(side);
      cudaEventDestroy(ev_x);
      cudaEventDestroy(ev_copied);
      side = nullptr;
    }
    ws.release();
    tcws.release();
    xws.release();
    prof.release();
  }
};

}  // namespace fks

using namespace fks;

struct fks_ctx {
  int device;
};

// K and M of a general sparse operator on the device: union pattern, K and M
// values per entry (fp64 and fp32), diagonals for the Jacobi preconditioner.
struct CsrDev {
  int64_t nnz = 0;
  int64_t* sell = nullptr;  // sliced ELL layout of the union pattern (CsrView)
  int32_t* len = nullptr;
  int32_t* col = nullptr;
  double *kv = nullptr, *mv = nullptr, *dk = nullptr, *dm = nullptr;
  float *kv32 = nullptr, *mv32 = nullptr;
  std::vector<double> dk_h, dm_h;  // host copies of the diagonals
  // host copies of the union pattern and values (the AMG setup reads them)
  std::vector<int64_t> rowptr_h;
  std::vector<int32_t> col_h;
  std::vector<double> kv_h, mv_h;
  template <typename T>
  fks::CsrView<T> view(int64_t n) const {
    fks::CsrView<T> v;
    v.n = n;
    v.sell = sell;
    v.len = len;
    v.col = col;
    if constexpr (sizeof(T) == 8) { v.kv = kv; v.mv = mv; } else { v.kv = kv32; v.mv = mv32; }
    return v;
  }
};

// Smoothed-aggregation AMG of a CSR operator: parameters, the aggregates
// (fixed by the first build), and the device hierarchies built so far, one
// per (tau, cycle precision).
struct AmgEntry {
  fks_c128 tau;
  int prec;
  std::vector<void*> mem;
  std::vector<unsigned char> lv;  // AmgLevel<T> of every level: rows of a solve's device table
};

struct AmgState {
  bool on = false;
  int max_levels = 10, nu = 2;
  int64_t max_coarse = 256;
  int gen = 0;                    // changes with the parameters (part of the graph key)
  AmgAgg agg;
  std::vector<int64_t> sizes, nnz, pnnz;  // per level: unknowns, entries of A and of P
  std::vector<AmgEntry> cache;
  std::mutex mu;
  void clear() {
    if (!cache.empty()) cudaDeviceSynchronize();  // no launch may still read a hierarchy
    for (auto& e : cache)
      for (void* p : e.mem) cudaFree(p);
    cache.clear();
    agg = AmgAgg{};
    sizes.clear();
    nnz.clear();
    pnnz.clear();
  }
};

struct fks_op {
  fks_ctx* ctx;
  int dim;   // 2 or 3 for grid operators, 0 for CSR operators
  bool csr = false;
  CsrDev cd;
  AmgState amg;
  int nx, ny, nz;
  int64_t n;
  uint32_t mask;
  double* cond_d = nullptr;  // grid operators: cell conductivity (device), for the sensitivities
  std::vector<LevelHost> levels;
  std::vector<LevelHost> levels_bf;  // the same levels with fp32 coefficients replaced by their bf16 roundings
  Lane lane0;  // workspace, graph and instrumentation of fks_solve / fks_precond_apply
  // 2D levels with at most this many cells use the fused tile kernels
  // ([0] complex128 cycles, [1] complex64 cycles); set by fks_op_autotune
  int64_t fuse_max[2] = {65536, INT64_MAX};
  // fused 2D levels with at most this many cells use 16 x 16 tiles (else 32 x 32)
  int64_t tile16_max[2] = {16384, 16384};
  // ... and with at most this many, 8 x 8 tiles (more CTAs on small levels)
  int64_t tile8_max[2] = {0, 0};
  // levels with at most this many cells run in the single-block tail kernel
  int64_t tail_max[2] = {256, 256};
  // from the first level with at most this many cells (and a cluster layout)
  // down, the V-cycle runs in the cluster kernel instead of the tail (0: off)
  int64_t cluster_max[2] = {0, 0};
  int64_t coop_max[2] = {0, 0};       // cooperative lower cycle from the first level <= this (0: off)
  // planes per block of the fused 3D level kernels, per level (0: the whole level)
  int zchunk[2][MAX_LEVELS] = {{16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16},
                               {16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16}};
};

namespace fks {

static bool prec_ok(int p) { return p == FKS_PREC_FP64 || p == FKS_PREC_MIXED || p == FKS_PREC_MIXED_BF16; }

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void copy_in(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return;
  CK(cudaMemcpyAsync(dst, src, bytes, is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
}
static void copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0 || !dst) return;
  CK(cudaMemcpyAsync(dst, src, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
}

// Shapes of the multigrid levels: axis a halves while n_a is even and > 4.
// Multigrid levels: an axis halves while its cell count is even and > 4. With
// `ragged`, an odd axis > 4 also halves (to (n + 1) / 2 cells, the last coarse
// cell having one child) while the level has more than MAX_COARSE cells; the
// operator takes the ragged hierarchy only when the even one ends above
// MAX_COARSE cells (the largest coarsest level solved exactly).
static std::vector<LevelHost> level_shapes(int nx, int ny, int nz, const double h[3], bool ragged) {
  std::vector<LevelHost> L;
  LevelHost l{};
  l.nx = nx; l.ny = ny; l.nz = nz;
  l.h[0] = h[0]; l.h[1] = h[1]; l.h[2] = h[2];
  while (true) {
    l.n = (int64_t)l.nx * l.ny * l.nz;
    const bool big = ragged && l.n > MAX_COARSE;
    l.rx = (l.nx > 4 && (l.nx % 2 == 0 || big)) ? 2 : 1;
    l.ry = (l.ny > 4 && (l.ny % 2 == 0 || big)) ? 2 : 1;
    l.rz = (l.nz > 4 && (l.nz % 2 == 0 || big)) ? 2 : 1;
    L.push_back(l);
    if (l.rx == 1 && l.ry == 1 && l.rz == 1) break;
    LevelHost c{};
    c.nx = (l.nx + l.rx - 1) / l.rx; c.ny = (l.ny + l.ry - 1) / l.ry; c.nz = (l.nz + l.rz - 1) / l.rz;
    c.h[0] = l.h[0] * l.rx; c.h[1] = l.h[1] * l.ry; c.h[2] = l.h[2] * l.rz;
    l = c;
    if ((int)L.size() >= MAX_LEVELS) break;
  }
  return L;
}

// ------------------------------------------------------------------ solve state
// Hooks of one cycle of a restarted solve (solve_restarted) into solve_impl.
struct RestartIO {
  const double* tol_shift;  // host [n_f * n_rhs]: each shift's tolerance, relative to its source's ||b||
  z64* coef;                // host out [n_f * n_rhs]: FFOM residual coefficient c at each shift's freeze step
  double* beta;             // host out [n_rhs]: ||b|| of each source
  int32_t* steps;           // host out [n_rhs]: Arnoldi steps taken
  z64* v_next;              // device out [n * n_rhs]: v_{k+1} after the last step, the common residual direction
  int reuse_setup;          // the workspace still holds this operator's preconditioner setup for these taus
};

struct Solve {
  fks_op* op;
  Lane* lane;
  cudaStream_t s;
  int nslot, n_f, n_tau, m, sched_len, precision, variant;
  int64_t n;
  double tol, eps;
  int max_cycles;
  bool replay;
  SlotState* st;
  SlotState* st_host;  // pinned mirror
  z64 *b, *sigma, *taus, *V, *Z, *w, *H, *taus_k, *h12, *mdpart, *g, *rs, *R, *Y, *X;
  z32* V32 = nullptr;  // complex64 copy of the basis (mixed precision), or null
  // continuous batching (server): steps left in a launch of the step loop, and
  // per-slot stop flags; null for fks_solve
  bool batching = false;
  int32_t* budget = nullptr;
  int32_t* stopv = nullptr;
  int32_t* tcerr = nullptr;  // the tensor-core assembly's error flag of a server batch
  double *pn, *rc, *est, *bnd, *dpart, *npart, *mpart, *wpart, *tpart, *tres;
  double* alpha;   // Prop. 3's alpha per (source, shift) at its freeze step
  double* tolv;    // per-shift tolerances of a restart cycle (used when tolv_on)
  z64* rcoef;      // FFOM residual coefficient per shift at its freeze step (restart cycles)
  bool tolv_on = false;
  int32_t *cyc, *sst, *mj, *sched, *rep_cyc, *rep_mj, *singular, *flags, *counter, *bcount;
  // multigrid, cycle precision
  std::vector<void*> f, z, z2, invd;
  void* cinv;      // coarse inverse in cycle precision
  z64* cwork;      // dense coarse matrices
  z64* cinv64;
  // CSR operators: BiCGSTAB cycle work vectors (cycle precision), scalars, Jacobi diagonals
  int inner_steps = 8;
  double relax = 0.0;  // relaxed inner tolerance constant (0: fixed eps)
  void* bv[9] = {};        // e, r, rh, p, v, ph, s, sh, t
  void* dinv = nullptr;    // [n_tau][n]
  // AMG-preconditioned cycles: device table [n_tau][L] and per-level vectors
  bool amg = false;
  int amg_L = 0;
  void* amg_tab = nullptr;
  std::vector<unsigned char> amg_table;  // host image of the table
  void *amg_f[AMG_MAX_LEVELS] = {}, *amg_x[AMG_MAX_LEVELS] = {}, *amg_y[AMG_MAX_LEVELS] = {},
       *amg_r[AMG_MAX_LEVELS] = {};
  BcgScal* bsc = nullptr;
  double* bpart = nullptr;
  int ndef = 0;            // blocks of the defect kernel (partials per slot)
  z64* diag64 = nullptr;           // finest level: K_cc + tau M_cc per distinct tau (fp64)
  unsigned char* tblob = nullptr;  // tail coefficients per tau in the shared-memory layout
  size_t tblob_bytes = 0;
  int tcoef0 = 0;
  unsigned char* cblob = nullptr;  // cluster kernel: band coefficients per tau and CTA
  bool capturing = false;  // enqueueing into a graph: no event timing
  // server batches hold this lock for their host-side CUDA calls and release it
  // only while they wait for their step-loop graph to finish
  std::unique_lock<std::mutex>* api_lock = nullptr;
};

// The bf16-smoother option: the V-cycle runs on op->levels_bf (coefficients
// rounded to bf16; bf16 storage for the per-level smoother and restriction).
static bool bf16_of(const Solve& S) { return S.precision == FKS_PREC_MIXED_BF16 && !S.op->csr; }
static const std::vector<LevelHost>& cycle_levels(const Solve& S) {
  return bf16_of(S) ? S.op->levels_bf : S.op->levels;
}

template <typename VT>
static BcgVecs<VT> bcg_vecs(Solve& S) {
  BcgVecs<VT> B;
  B.f = (cx<VT>*)S.f[0];
  cx<VT>** d[9] = {&B.e, &B.r, &B.rh, &B.p, &B.v, &B.ph, &B.s, &B.sh, &B.t};
  for (int i = 0; i < 9; ++i) *d[i] = (cx<VT>*)S.bv[i];
  return B;
}

static int defect_partials(const fks_op* op) {
  return op->csr ? csr_blocks(op->n) : defect_blocks(op->levels[0]);
}

#define PROF(cls, lvl, by, fl, call)                                           \
  do {                                                                        \
    S.lane->prof.begin(S.capturing ? -1 : (cls), (lvl), (by), (fl), S.s);     \
    call;                                                                     \
    S.lane->prof.end(S.s);                                                    \
  } while (0)

// First level handled by the single-block tail V-cycle: the first with at most
// `tmax` cells (the operator's tail threshold for the cycle precision, chosen
// by fks_op_autotune; the tail runs on one SM, larger levels spread over SMs
// in tile kernels).
template <typename VT>
static int tail_level(const std::vector<LevelHost>& Ls, int64_t tmax) {
  for (size_t l = 0; l < Ls.size(); ++l)
    if (Ls[l].n <= tmax) return (int)l;
  return (int)Ls.size() - 1;
}

template <typename VT>
static int64_t tail_max_of(const fks_op* op) { return op->tail_max[sizeof(VT) == 8 ? 0 : 1]; }

// First level of the cluster V-cycle for threshold cmax: the first level with
// at most cmax cells whose cluster layout applies, else the next coarser one
// that does; -1 when off or none applies. P / smem receive the layout.
template <typename VT>
static int cluster_level_for(const std::vector<LevelHost>& Ls, int64_t cmax, ClusterParams<VT>* P = nullptr,
                             size_t* smem = nullptr) {
  if (cmax <= 0) return -1;
  for (size_t l = 0; l + 1 < Ls.size(); ++l) {
    if (Ls[l].n > cmax) continue;
    ClusterParams<VT> Q;
    size_t sm = 0;
    if (cluster_layout<VT>(Ls, (int)l, &Q, &sm)) {
      if (P) *P = Q;
      if (smem) *smem = sm;
      return (int)l;
    }
  }
  return -1;
}

template <typename VT>
static int cluster_level(const fks_op* op, ClusterParams<VT>* P = nullptr, size_t* smem = nullptr) {
  if (op->csr) return -1;
  return cluster_level_for<VT>(op->levels, op->cluster_max[sizeof(VT) == 8 ? 0 : 1], P, smem);
}

constexpr size_t TAIL_SMEM_LIMIT = 220 * 1024;

// Shared memory of the tail kernel: f and z of every tail level, then (when it
// fits) each level's coefficients (faces, storage, inverse diagonals for the
// current tau). Returns the bytes; `coef_byte` receives each level's offset.
template <typename VT>
static size_t tail_layout(const std::vector<LevelHost>& Ls, int lt, bool staged, std::vector<int>* coef_byte) {
  size_t e = 0;
  for (size_t l = lt; l < Ls.size(); ++l) e += 2 * (size_t)Ls[l].n;
  size_t bytes = e * sizeof(cx<VT>);
  if (coef_byte) coef_byte->assign(Ls.size(), -1);
  if (!staged) return bytes;
  for (size_t l = lt; l < Ls.size(); ++l) {
    const LevelHost& L = Ls[l];
    size_t realn = face_count(L, 0) + face_count(L, 1) + (L.nz > 1 ? face_count(L, 2) : 0) + L.n;
    realn = (realn + 3) & ~(size_t)3;
    bytes = (bytes + 15) & ~(size_t)15;
    if (coef_byte) (*coef_byte)[l] = (int)bytes;
    bytes += realn * sizeof(VT) + (size_t)L.n * sizeof(cx<VT>);
  }
  return (bytes + 15) & ~(size_t)15;
}

template <typename VT>
static bool tail_staged(const std::vector<LevelHost>& Ls, int lt) {
  return tail_layout<VT>(Ls, lt, true, nullptr) <= TAIL_SMEM_LIMIT;
}

template <typename VT>
static size_t tail_smem(const std::vector<LevelHost>& Ls, int lt) {
  return tail_layout<VT>(Ls, lt, tail_staged<VT>(Ls, lt), nullptr);
}

// Shared memory of the tail launch from level lt; *pairs = 1 when it is the
// register-resident 2D kernel (coefficients staged, the levels qualify and the
// coarsest inverse, staged at *ainv_off, fits as well).
template <typename VT>
static size_t tail_launch_smem(const std::vector<LevelHost>& Ls, int lt, int* pairs = nullptr,
                               int* ainv_off = nullptr) {
  const size_t b = tail_smem<VT>(Ls, lt);
  if (pairs) *pairs = 0;
  if (ainv_off) *ainv_off = 0;
  if (!tail_staged<VT>(Ls, lt) || !tail2d_ok(Ls, lt)) return b;
  const size_t nc = (size_t)Ls.back().n;
  const size_t a = (b + 15) & ~(size_t)15;
  const size_t b2 = a + nc * nc * sizeof(cx<VT>);
  if (b2 > TAIL_SMEM_LIMIT) return b;
  if (pairs) *pairs = 1;
  if (ainv_off) *ainv_off = (int)a;
  return b2;
}

// Bytes per tau of the tail's staged coefficients and their shared-memory
// offset (0 bytes when the tail reads its coefficients from global memory).
template <typename VT>
static size_t tail_blob_bytes(const std::vector<LevelHost>& Ls, int64_t tmax, int* coef0) {
  const int lt = tail_level<VT>(Ls, tmax);
  std::vector<int> cb;
  if (!tail_staged<VT>(Ls, lt)) {
    *coef0 = 0;
    return 0;
  }
  size_t total = tail_layout<VT>(Ls, lt, true, &cb);
  *coef0 = cb[lt];
  return total - (size_t)cb[lt];
}

// One V-cycle on f[0]; returns the buffer holding the level-0 correction, or
// null when the finest level's post-smoothing kernel already added it to
// column k - 1 of Zk (given with its strides; Zk null: never).
template <typename VT>
static cx<VT>* vcycle(Solve& S, z64* Zk = nullptr, int64_t vsZk = 0, int64_t zcol = 0) {
  const auto& Ls = cycle_levels(S);
  const int bf = bf16_of(S) ? 1 : 0;
  int nl = (int)Ls.size();
  ClusterParams<VT> CP{};
  size_t csmem = 0;
  const int lc = cluster_level<VT>(S.op, &CP, &csmem);
  // first level of the single-launch lower part: the cluster kernel's, else the tail's
  int lt = lc >= 0 ? lc : tail_level<VT>(Ls, tail_max_of<VT>(S.op));
  // or the cooperative lower cycle's, when it is on and starts above the tail
  int lco = -1;
  const int64_t cmx = S.op->coop_max[sizeof(VT) == 8 ? 0 : 1];
  if (lc < 0 && cmx > 0) {
    for (int l = 1; l < lt; ++l)
      if (Ls[l].n <= cmx) {
        lco = l;
        break;
      }
    if (lco >= 0 && coop_capacity_vcycle<VT>() <= 0) lco = -1;
  }
  const int lp = lco >= 0 ? lco : lt;
  cudaStream_t s = S.s;
  auto F = [&](int l) { return (cx<VT>*)S.f[l]; };
  auto Zl = [&](int l) { return (cx<VT>*)S.z[l]; };
  auto I = [&](int l) { return (const cx<VT>*)S.invd[l]; };
  const double cv = sizeof(cx<VT>), rv = sizeof(VT), d = S.op->dim, ns = S.nslot;
  // algorithmic bytes / flops per launch (per level), see the class list in fks.h
  auto smooth_b = [&](const LevelHost& L, int zs) {
    return zs ? ns * L.n * 1.5 * cv : ns * L.n * (2 * cv + d * rv);
  };
  auto smooth_f = [&](const LevelHost& L, int zs) { return zs ? ns * L.n * 3.0 : ns * L.n * 0.5 * (8 * d + 6); };
  const int64_t fmax = S.op->fuse_max[sizeof(VT) == 8 ? 0 : 1];
  const int64_t t16 = S.op->tile16_max[sizeof(VT) == 8 ? 0 : 1];
  const int64_t t8 = S.op->tile8_max[sizeof(VT) == 8 ? 0 : 1];
  auto tile_of = [&](const LevelHost& L) { return L.n <= t8 ? 8 : (L.n <= t16 ? 16 : 32); };
  const int pix = sizeof(VT) == 8 ? 0 : 1;
  for (int l = 0; l < lp; ++l) {
    const LevelHost& L = Ls[l];
    if (fused_level_ok(L) && L.n <= fmax) {
      PROF(FKS_K_PRE2D, l, ns * (L.n * (3 * cv + (d + 1) * rv) + cv * Ls[l + 1].n),
           ns * L.n * (2 * (8 * d + 6) + 8 * d + 10),
           launch_pre2d<VT>(L, Ls[l + 1], S.st, I(l), S.taus, F(l), Zl(l), L.n, F(l + 1), Ls[l + 1].n, S.nslot,
                            tile_of(L), s));
      continue;
    }
    if (fused3d_level_ok(L) && L.n <= fmax) {
      PROF(FKS_K_PRE3D, l, ns * (L.n * (3 * cv + (d + 1) * rv) + cv * Ls[l + 1].n),
           ns * L.n * (2 * (8 * d + 6) + 8 * d + 10),
           launch_pre3d<VT>(L, S.st, I(l), S.taus, F(l), Zl(l), L.n, F(l + 1), Ls[l + 1].n, S.nslot, tile_of(L),
                            S.op->zchunk[pix][l], s));
      continue;
    }
    for (int r = 0; r < NU1; ++r) {
      int zs = r == 0 ? 1 : 0;
      PROF(FKS_K_SMOOTH, l, smooth_b(L, zs), smooth_f(L, zs),
           launch_gs<VT>(L, S.st, I(l), F(l), Zl(l), L.n, S.nslot, 0, zs, s, nullptr, 0, 0, bf));
      PROF(FKS_K_SMOOTH, l, smooth_b(L, 0), smooth_f(L, 0),
           launch_gs<VT>(L, S.st, I(l), F(l), Zl(l), L.n, S.nslot, 1, 0, s, nullptr, 0, 0, bf));
    }
    PROF(FKS_K_RESTRICT, l, ns * (L.n * (2 * cv + (d + 1) * rv) + cv * Ls[l + 1].n), ns * L.n * (8 * d + 10),
         launch_residual_restrict<VT>(L, Ls[l + 1], S.st, S.taus, F(l), Zl(l), L.n, F(l + 1), Ls[l + 1].n, S.nslot,
                                      s, bf));
  }
  if (lco >= 0) {
    // levels lco .. coarsest in one cooperative launch
    CoopParams<VT> P{};
    P.nlev = nl - lco;
    double tb = 0, tf = 0;
    int64_t most = 0;
    for (int l = lco; l < nl; ++l) {
      const int i = l - lco;
      P.L[i] = view<VT>(Ls[l]);
      P.invd[i] = I(l);
      P.f[i] = F(l);
      P.z[i] = Zl(l);
      P.rx[i] = Ls[l].rx; P.ry[i] = Ls[l].ry; P.rz[i] = Ls[l].rz;
      tb += Ls[l].n * (8 * cv + d * rv);
      tf += Ls[l].n * (8 * d + 6) * 4;
      most = std::max<int64_t>(most, Ls[l].n);
    }
    const LevelHost& C = Ls[nl - 1];
    P.Ainv = (const cx<VT>*)S.cinv;
    P.nc = (int)C.n;
    P.mask = S.op->mask;
    P.taus = S.taus;
    P.nslot = S.nslot;
    tb += cv * C.n * C.n;
    tf += 8.0 * C.n * C.n;
    const int blocks = (int)std::min<int64_t>((most * S.nslot + 255) / 256, INT_MAX);
    bool ok = false;
    PROF(FKS_K_COOP, lco, ns * tb, ns * tf, ok = launch_coop_vcycle<VT>(P, S.st, blocks, s));
    if (!ok) throw CudaError{cudaErrorLaunchFailure, "cooperative lower V-cycle launch"};
  } else if (lc >= 0) {
    // levels lc .. coarsest in one cluster per slot
    CP.mask = S.op->mask;
    CP.f_in = F(lc);
    CP.z_out = Zl(lc);
    CP.vs = Ls[lc].n;
    CP.blob = S.cblob;
    CP.taus = S.taus;
    double tb = 0, tf = 0;
    for (int l = lc; l < nl; ++l) {
      tb += Ls[l].n * (8 * cv + d * rv);
      tf += Ls[l].n * (8 * d + 6) * 4;
    }
    const int64_t nc = Ls[nl - 1].n;
    tb += cv * nc * nc;
    tf += 8.0 * nc * nc;
    PROF(FKS_K_CLUSTER, lc, ns * tb, ns * tf, launch_cluster_vcycle<VT>(CP, csmem, S.st, S.nslot, s));
  } else {
    // levels lt .. coarsest in one block per slot
    TailParams<VT> P{};
    P.nlev = nl - lt;
    P.staged = tail_staged<VT>(Ls, lt) ? 1 : 0;
    std::vector<int> cbyte;
    tail_layout<VT>(Ls, lt, P.staged != 0, &cbyte);
    int off = 0;
    double tb = 0, tf = 0;
    for (int l = lt; l < nl; ++l) {
      TailLevel<VT>& T = P.lev[l - lt];
      T.L = view<VT>(Ls[l]);
      T.rx = Ls[l].rx; T.ry = Ls[l].ry; T.rz = Ls[l].rz;
      T.invd = I(l);
      T.off = off;
      T.cbyte = cbyte[l];
      off += 2 * (int)Ls[l].n;
      tb += Ls[l].n * (8 * cv + d * rv);
      tf += Ls[l].n * (8 * d + 6) * 4;
    }
    const LevelHost& C = Ls[nl - 1];
    P.Ainv = (const cx<VT>*)S.cinv;
    P.nc = (int)C.n;
    P.mask = S.op->mask;
    P.f_in = F(lt);
    P.z_out = Zl(lt);
    P.vs = Ls[lt].n;
    P.taus = S.taus;
    P.blob = S.tblob;
    P.blob_bytes = (int)S.tblob_bytes;
    P.coef0 = S.tcoef0;
    tb += cv * C.n * C.n;
    tf += 8.0 * C.n * C.n;
    const size_t tsm = tail_launch_smem<VT>(Ls, lt, &P.pairs, &P.ainv_off);
    if (!P.blob) P.pairs = 0;
    PROF(FKS_K_TAIL, lt, ns * tb, ns * tf, launch_tail<VT>(P, tsm, S.st, S.nslot, s));
  }
  cx<VT>* zfin = Zl(lp);  // final correction of the level below
  for (int l = lp - 1; l >= 0; --l) {
    const LevelHost& L = Ls[l];
    if (fused_level_ok(L) && L.n <= fmax) {
      cx<VT>* out = (cx<VT>*)S.z2[l];
      const bool add_to_zk = l == 0 && Zk;
      PROF(FKS_K_POST2D, l, ns * (L.n * (4 * cv + d * rv) + cv * Ls[l + 1].n),
           ns * L.n * (18 + 2 * (8 * d + 6)),
           launch_post2d<VT>(L, Ls[l + 1], S.op->mask, S.st, I(l), F(l), Zl(l), out, L.n, zfin, Ls[l + 1].n,
                             S.nslot, tile_of(L), s, add_to_zk ? Zk : nullptr, vsZk, zcol));
      zfin = add_to_zk ? nullptr : out;
      continue;
    }
    if (fused3d_level_ok(L) && L.n <= fmax) {
      cx<VT>* out = (cx<VT>*)S.z2[l];
      const bool add_to_zk = l == 0 && Zk;
      PROF(FKS_K_POST3D, l, ns * (L.n * (4 * cv + d * rv) + cv * Ls[l + 1].n),
           ns * L.n * (18 + 2 * (8 * d + 6)),
           launch_post3d<VT>(L, S.op->mask, S.st, I(l), F(l), Zl(l), out, L.n, zfin, Ls[l + 1].n, S.nslot,
                             tile_of(L), S.op->zchunk[pix][l], s, add_to_zk ? Zk : nullptr, vsZk, zcol));
      zfin = add_to_zk ? nullptr : out;
      continue;
    }
    PROF(FKS_K_PROLONG, l, ns * (2 * cv * L.n + cv * Ls[l + 1].n), ns * L.n * (4.0 * (1 << S.op->dim) + 2),
         launch_prolong_add<VT>(L, Ls[l + 1], S.op->mask, S.st, zfin, Ls[l + 1].n, Zl(l), L.n, S.nslot, s));
    // on the finest level the last half sweep also adds the correction to z_k
    const bool add_to_zk = l == 0 && Zk;
    for (int r = 0; r < NU2; ++r) {
      PROF(FKS_K_SMOOTH, l, smooth_b(L, 0), smooth_f(L, 0),
           launch_gs<VT>(L, S.st, I(l), F(l), Zl(l), L.n, S.nslot, 1, 0, s, nullptr, 0, 0, bf));
      const bool last = add_to_zk && r == NU2 - 1;
      PROF(FKS_K_SMOOTH, l, smooth_b(L, 0) + (last ? ns * L.n * 32.0 : 0.0), smooth_f(L, 0) + (last ? ns * L.n * 2.0 : 0.0),
           launch_gs<VT>(L, S.st, I(l), F(l), Zl(l), L.n, S.nslot, 0, 0, s, last ? Zk : nullptr, vsZk, zcol, bf));
    }
    zfin = add_to_zk ? nullptr : Zl(l);
  }
  return zfin;
}

static bool any_inner_running(Solve& S) {
  CK(cudaMemcpyAsync(S.st_host, S.st, sizeof(SlotState) * S.nslot, cudaMemcpyDeviceToHost, S.s));
  CK(cudaStreamSynchronize(S.s));
  for (int i = 0; i < S.nslot; ++i)
    if (S.st_host[i].active && !S.st_host[i].inner_done) return true;
  return false;
}

static bool any_active(Solve& S) {
  CK(cudaMemcpyAsync(S.st_host, S.st, sizeof(SlotState) * S.nslot, cudaMemcpyDeviceToHost, S.s));
  CK(cudaStreamSynchronize(S.s));
  for (int i = 0; i < S.nslot; ++i)
    if (S.st_host[i].active) return true;
  return false;
}

// ------------------------------------------------------------------ sections of a step
// Each section only enqueues kernels on S.s and reads nothing back, so that it
// can be captured into a graph; `use_cond` makes the deciding kernel set the
// given graph loop condition.

// First defect of the inner solve of step k: r = v_k (z = 0), ||v_k||.
template <typename VT>
static void sec_inner_first(Solve& S, const z64* V, int64_t vsV, z64* Z, int64_t vsZ, int use_cond,
                            cudaGraphConditionalHandle hin) {
  cx<VT>* f0 = (cx<VT>*)S.f[0];
  const int32_t* rc = S.replay ? S.rep_cyc : nullptr;
  const int64_t N = S.n;
  const double cv = sizeof(cx<VT>), ns = S.nslot, n = N;
  if (S.op->csr) {
    PROF(FKS_K_DEFECT, 0, ns * n * (16 + cv), ns * n * 4.0,
         launch_csr_defect<VT>(S.op->cd.view<double>(N), S.st, S.taus, V, vsV, Z, vsZ, N, 1, f0, N, S.dpart,
                               S.nslot, S.s));
    PROF(-1, -1, 0, 0,
         launch_inner_decide(S.st, S.nslot, S.dpart, S.ndef, 1, S.eps, S.max_cycles, rc, S.m, use_cond, hin, S.flags,
                             S.counter, S.s, S.relax, S.tol));
  } else {
    // defect and decision in one launch
    PROF(FKS_K_DEFECT, 0, ns * n * (16 + cv), ns * n * 4.0,
         launch_defect_decide<VT>(S.op->levels[0], S.st, S.taus, S.diag64, V, vsV, Z, vsZ, N, 1, f0, N, S.dpart, S.eps,
                                  S.max_cycles, rc, S.m, use_cond, hin, S.flags, S.counter, S.bcount, S.nslot,
                                  S.relax, S.tol, S.s));
  }
}

// One BiCGSTAB cycle of a CSR operator's inner solve; returns its result e.
template <typename VT>
static cx<VT>* bicgstab_cycle(Solve& S) {
  const int64_t N = S.n;
  const double cv = sizeof(cx<VT>), rv = sizeof(VT), ns = S.nslot, n = N, nnz = S.op->cd.nnz;
  const double st = S.inner_steps;
  // per step: two products over the union pattern (column + K + M per entry and
  // the gathered vector), and about 24 vector passes
  const double by = ns * (n * cv * 8 + st * (2 * (nnz * (4 + 2 * rv + cv) + 8 * n) + 24 * n * cv));
  const double fl = ns * st * (2 * nnz * 10 + n * 60);
  BcgVecs<VT> B = bcg_vecs<VT>(S);
  int extra = 0;
  if (S.amg) {
    const AmgState& M = S.op->amg;
    AmgRun<VT> R{};
    R.tab = (const AmgLevel<VT>*)S.amg_tab;
    R.L = S.amg_L;
    R.nu = M.nu;
    // per step two V-cycles: on every level but the coarsest 2 nu products with
    // A_l (nu - 1 sweeps and the residual down, nu sweeps up; the first sweep
    // is elementwise, done by the kernel that writes the level's right-hand
    // side), P and P^T, and the vectors they stream; the coarsest level's dense
    // inverse. Flops count a complex multiply-add as 8.
    double vb = 0.0, vf = 0.0;
    for (int l = 0; l < S.amg_L; ++l) {
      const double nl = (double)M.sizes[l], al = (double)M.nnz[l];
      if (l + 1 < S.amg_L) {
        const double pl = (double)M.pnnz[l], passes = 2.0 * M.nu;
        vb += passes * (al * (12 + cv) + nl * 4 * cv) + 2 * (pl * (12 + cv) + nl * 2 * cv);
        vf += passes * al * 8 + 2 * pl * 8;
      } else {
        vb += nl * nl * cv + 2 * nl * cv;
        vf += nl * nl * 8;
      }
    }
    const double aby = ns * (n * cv * 8 + st * (2 * (nnz * (4 + 2 * rv + cv) + 8 * n) + 24 * n * cv + 2 * vb));
    const double afl = ns * st * (2 * nnz * 10 + n * 60 + 2 * vf);
    for (int l = 0; l < S.amg_L; ++l) {
      R.n[l] = M.sizes[l];
      R.f[l] = (cx<VT>*)S.amg_f[l];
      R.x[l] = (cx<VT>*)S.amg_x[l];
      R.y[l] = (cx<VT>*)S.amg_y[l];
      R.r[l] = (cx<VT>*)S.amg_r[l];
    }
    PROF(FKS_K_BICGSTAB, 0, aby, afl,
         launch_bcg_cycle_amg<VT>(S.op->cd.view<VT>(N), S.st, S.taus, B, R, S.bsc, S.bpart, S.inner_steps, S.nslot,
                                  S.s, &extra));
  } else {
    PROF(FKS_K_BICGSTAB, 0, by, fl,
         launch_bcg_cycle<VT>(S.op->cd.view<VT>(N), S.st, S.taus, B, (const cx<VT>*)S.dinv, S.bsc, S.bpart,
                              S.inner_steps, S.nslot, S.s, &extra));
  }
  S.lane->prof.all_launches += extra - 1;
  return B.e;
}

// K + tau M on the entries where K or M is nonzero (and the diagonal): level 0
// of the AMG hierarchy, whose pattern is the strength graph
static AmgCsr amg_level0(const fks_op* op, fks_c128 tau) {
  const CsrDev& C = op->cd;
  AmgCsr A;
  A.n = A.m = op->n;
  A.rp.assign(op->n + 1, 0);
  for (int64_t i = 0; i < op->n; ++i) {
    for (int64_t q = C.rowptr_h[i]; q < C.rowptr_h[i + 1]; ++q) {
      const double k = C.kv_h[q], m = C.mv_h[q];
      if (C.col_h[q] != i && k == 0.0 && m == 0.0) continue;
      A.ci.push_back(C.col_h[q]);
      A.v.push_back(mk(k + tau.re * m, tau.im * m));
    }
    A.rp[i + 1] = (int64_t)A.ci.size();
  }
  return A;
}

// The hierarchies of the n_tau taus in cycle precision VT (built on first use,
// then cached on the operator); `table` receives their levels, tau after tau.
// Returns "" or an error message.
template <typename VT>
static std::string amg_ensure(fks_op* op, const fks_c128* tau, int n_tau, std::vector<AmgLevel<VT>>* table,
                              double* setup_ms = nullptr) {
  AmgState& M = op->amg;
  std::lock_guard<std::mutex> lock(M.mu);
  const int prec = sizeof(VT) == 8 ? FKS_PREC_FP64 : FKS_PREC_MIXED;
  const auto t0 = std::chrono::steady_clock::now();
  table->clear();
  for (int q = 0; q < n_tau; ++q) {
    int hit = -1;
    for (size_t e = 0; e < M.cache.size(); ++e)
      if (M.cache[e].prec == prec && M.cache[e].tau.re == tau[q].re && M.cache[e].tau.im == tau[q].im) hit = (int)e;
    if (hit < 0) {
      AmgHost h;
      std::string err = amg_build(amg_level0(op, tau[q]), M.max_levels, M.max_coarse, &M.agg, &h);
      if (!err.empty()) return err;
      if (M.sizes.empty())
        for (const auto& L : h.lv) {
          M.sizes.push_back(L.A.n);
          M.nnz.push_back((int64_t)L.A.ci.size());
          M.pnnz.push_back((int64_t)L.P.ci.size());
        }
      AmgEntry ne;
      ne.tau = tau[q];
      ne.prec = prec;
      std::vector<AmgLevel<VT>> lv;
      cudaError_t ce = amg_upload<VT>(h, ne.mem, lv);
      if (ce != cudaSuccess) {
        for (void* p : ne.mem) cudaFree(p);
        throw CudaError{ce, "AMG upload"};
      }
      ne.lv.resize(sizeof(AmgLevel<VT>) * lv.size());
      std::memcpy(ne.lv.data(), lv.data(), ne.lv.size());
      M.cache.push_back(std::move(ne));
      hit = (int)M.cache.size() - 1;
    }
    const AmgEntry& E = M.cache[hit];
    const size_t nl = E.lv.size() / sizeof(AmgLevel<VT>);
    const size_t at = table->size();
    table->resize(at + nl);
    std::memcpy(table->data() + at, E.lv.data(), E.lv.size());
  }
  if (setup_ms)
    *setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return "";
}

// Before the carve of a CSR solve with AMG: the taus' hierarchies and the
// host image of the solve's table. Returns "" or an error message.
template <typename VT>
static std::string amg_prepare(Solve& S, const fks_c128* tau) {
  S.amg = S.op->csr && S.op->amg.on;
  if (!S.amg) return "";
  std::vector<fks_c128> th(S.n_tau);
  CK(cudaMemcpy(th.data(), tau, sizeof(fks_c128) * S.n_tau, cudaMemcpyDefault));
  std::vector<AmgLevel<VT>> tab;
  std::string err = amg_ensure<VT>(S.op, th.data(), S.n_tau, &tab);
  if (!err.empty()) return err;
  S.amg_L = (int)S.op->amg.sizes.size();
  S.amg_table.resize(sizeof(AmgLevel<VT>) * tab.size());
  std::memcpy(S.amg_table.data(), tab.data(), S.amg_table.size());
  return "";
}

// One inner cycle: z += V-cycle(r), r = v - (K + tau M) z, decide.
template <typename VT>
static void sec_inner_body(Solve& S, const z64* V, int64_t vsV, z64* Z, int64_t vsZ, int use_cond,
                           cudaGraphConditionalHandle hin) {
  cx<VT>* f0 = (cx<VT>*)S.f[0];
  const int32_t* rc = S.replay ? S.rep_cyc : nullptr;
  const int64_t N = S.n;
  const double cv = sizeof(cx<VT>), d = S.op->dim, ns = S.nslot, n = N;
  cx<VT>* e0 = S.op->csr ? bicgstab_cycle<VT>(S) : vcycle<VT>(S, Z, vsZ, N);
  if (e0)  // else the finest post-smoothing kernel already added the correction
    PROF(FKS_K_CORRECT, 0, ns * n * (cv + 32), ns * n * 2.0,
         launch_correct<VT>(S.st, Z, vsZ, N, e0, N, N, S.nslot, S.s));
  if (S.op->csr) {
    const double nnz = S.op->cd.nnz;
    PROF(FKS_K_DEFECT, 0, ns * (n * (40 + cv) + nnz * 20 + nnz * 16), ns * nnz * 10.0,
         launch_csr_defect<VT>(S.op->cd.view<double>(N), S.st, S.taus, V, vsV, Z, vsZ, N, 0, f0, N, S.dpart,
                               S.nslot, S.s));
    PROF(-1, -1, 0, 0,
         launch_inner_decide(S.st, S.nslot, S.dpart, S.ndef, 0, S.eps, S.max_cycles, rc, S.m, use_cond, hin, S.flags,
                             S.counter, S.s, S.relax, S.tol));
  } else {
    // defect and decision in one launch (the K diagonal is precomputed on this level)
    PROF(FKS_K_DEFECT, 0, ns * n * (32 + 8 * (d + 2) + cv), ns * n * (8 * d + 10),
         launch_defect_decide<VT>(S.op->levels[0], S.st, S.taus, S.diag64, V, vsV, Z, vsZ, N, 0, f0, N, S.dpart, S.eps,
                                  S.max_cycles, rc, S.m, use_cond, hin, S.flags, S.counter, S.bcount, S.nslot,
                                  S.relax, S.tol, S.s));
  }
}

// Inner solve of the current step, host-driven: z_k (column k-1 of Z) from v_k.
template <typename VT>
static void inner_solve(Solve& S, const z64* V, int64_t vsV, z64* Z, int64_t vsZ) {
  sec_inner_first<VT>(S, V, vsV, Z, vsZ, 0, 0);
  int guard = 0;
  while (any_inner_running(S)) {
    sec_inner_body<VT>(S, V, vsV, Z, vsZ, 0, 0);
    if (++guard > 100000) break;
  }
}

static void sec_step_begin(Solve& S) {
  PROF(-1, -1, 0, 0, launch_step_begin(S.st, S.nslot, S.sched, S.sched_len, S.taus, S.taus_k, S.m, S.s));
}

// After the inner solve: w = M z_k, CGS2, h_{k+1,k}, v_{k+1}, per-shift least
// squares, end-of-step test. `step` only sizes the launches in host-driven
// mode (graphs use m_max and let idle blocks exit).
static void sec_step_end(Solve& S, int step, int use_cond, cudaGraphConditionalHandle hout) {
  const int64_t n = S.n;
  const int m = S.m, n_f = S.n_f, n_rhs = S.nslot;
  const int64_t vsV = (int64_t)(m + 1) * n, vsZ = (int64_t)m * n;
  const double ns = n_rhs, nn = (double)n, kk = step;
  const int kmax = use_cond ? m : step;
  if (S.op->csr)
    PROF(-1, -1, 0, 0, launch_csr_mass(S.op->cd.view<double>(n), S.st, S.Z, vsZ, S.w, S.mpart, n_rhs, S.s));
  else
    PROF(-1, -1, 0, 0, launch_mass(S.st, S.op->levels[0].d64[3], S.Z, vsZ, S.w, n, S.mpart, n_rhs, S.s));
  // CGS2: two projections; pass p writes its coefficients to h12[slot][p]
  for (int pass = 0; pass < 2; ++pass) {
    z64* hp = S.h12 + pass * MAX_M;
    if (pass == 0 && S.V32)
      PROF(FKS_K_MDOT, -1, ns * (8 * nn * kk + 16 * nn), ns * 8 * nn * kk,
           launch_mdot32(S.st, S.V32, vsV, S.w, n, S.mdpart, kmax, n_rhs, S.s));
    else
      PROF(FKS_K_MDOT, -1, ns * 16 * nn * (kk + 1), ns * 8 * nn * kk,
           launch_mdot(S.st, S.V, vsV, S.w, n, S.mdpart, kmax, n_rhs, S.s));
    PROF(-1, -1, 0, 0, launch_hreduce(S.st, S.mdpart, n, hp, 2 * MAX_M, n_rhs, S.s));
    PROF(FKS_K_MAXPY, -1, ns * 16 * nn * (kk + 2), ns * 8 * nn * kk,
         launch_maxpy(S.st, S.V, vsV, hp, 2 * MAX_M, S.w, n, n_rhs, S.s));
  }
  PROF(-1, -1, 0, 0, launch_norm2_partial(S.st, 1, S.w, n, n, S.wpart, n_rhs, S.s));
  PROF(-1, -1, 0, 0,
       launch_arnoldi_finish(S.st, n_rhs, S.h12, S.wpart, S.mpart, norm_blocks(n), S.H, m, S.pn, S.cyc,
                             BREAKDOWN_RTOL, S.s));
  PROF(-1, -1, 0, 0, launch_new_v(S.st, S.w, n, S.H, m, S.V, vsV, n_rhs, S.s, S.V32));
  PROF(FKS_K_GIVENS, -1, ns * n_f * 48.0 * kk, ns * n_f * 26.0 * kk,
       launch_givens(S.st, n_f, m, S.sigma, S.H, S.taus_k, S.pn, S.tol, S.variant, S.replay ? S.rep_mj : nullptr,
                     S.g, S.rc, S.rs, S.R, S.Y, S.sst, S.mj, S.est, S.bnd, S.alpha, n_rhs, S.s,
                     S.tolv_on ? S.tolv : nullptr, S.tolv_on ? S.rcoef : nullptr));
  PROF(-1, -1, 0, 0, launch_step_end(S.st, n_rhs, m, use_cond, hout, S.s, S.budget));
}

// The loop over Arnoldi steps as one graph: outer WHILE (some source active) {
// step begin, first defect, inner WHILE (some inner solve running) { V-cycle,
// correct, defect, decide }, CGS2 ... end of step }. Kernel counts per section
// are returned for the launch count.
template <typename VT>
static void build_graph(Solve& S, cudaGraphExec_t* exec, int* outer_kernels, int* inner_kernels) {
  std::lock_guard<std::mutex> build_lock(g_build_mu);
  const int64_t n = S.n;
  const int m = S.m;
  const int64_t vsV = (int64_t)(m + 1) * n, vsZ = (int64_t)m * n;
  cudaStream_t user = S.s;
  cudaStream_t cs = nullptr;
  cudaGraph_t g = nullptr;
  int64_t saved = S.lane->prof.all_launches;
  try {
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle hout, hin;
    CK(cudaGraphConditionalHandleCreate(&hout, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams po = {};
    po.type = cudaGraphNodeTypeConditional;
    po.conditional.handle = hout;
    po.conditional.type = cudaGraphCondTypeWhile;
    po.conditional.size = 1;
    cudaGraphNode_t nout;
    CK(cudaGraphAddNode(&nout, g, nullptr, nullptr, 0, &po));
    cudaGraph_t body_out = po.conditional.phGraph_out[0];
    S.s = cs;
    S.capturing = true;
    int64_t c0 = S.lane->prof.all_launches;
    CK(cudaStreamBeginCaptureToGraph(cs, body_out, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    sec_step_begin(S);
    CK(cudaGraphConditionalHandleCreate(&hin, body_out, 0, 0));
    sec_inner_first<VT>(S, S.V, vsV, S.Z, vsZ, 1, hin);
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    CK(cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
    cudaGraphNodeParams pi = {};
    pi.type = cudaGraphNodeTypeConditional;
    pi.conditional.handle = hin;
    pi.conditional.type = cudaGraphCondTypeWhile;
    pi.conditional.size = 1;
    cudaGraphNode_t nin;
    CK(cudaGraphAddNode(&nin, body_out, deps, nullptr, ndeps, &pi));
    cudaGraph_t body_in = pi.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(cs, &nin, nullptr, 1, cudaStreamSetCaptureDependencies));
    sec_step_end(S, m, 1, hout);
    cudaGraph_t cap = nullptr;
    CK(cudaStreamEndCapture(cs, &cap));
    int64_t c1 = S.lane->prof.all_launches;
    CK(cudaStreamBeginCaptureToGraph(cs, body_in, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    sec_inner_body<VT>(S, S.V, vsV, S.Z, vsZ, 1, hin);
    CK(cudaStreamEndCapture(cs, &cap));
    int64_t c2 = S.lane->prof.all_launches;
    *outer_kernels = (int)(c1 - c0);
    *inner_kernels = (int)(c2 - c1);
    CK(cudaGraphInstantiate(exec, g, 0));
  } catch (...) {
    S.s = user;
    S.capturing = false;
    S.lane->prof.all_launches = saved;
    if (g) cudaGraphDestroy(g);
    if (cs) cudaStreamDestroy(cs);
    throw;
  }
  S.s = user;
  S.capturing = false;
  S.lane->prof.all_launches = saved;
  cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
}

// build_graph with programmatic dependent launches; if the capture or the
// instantiation refuses them, the process switches them off and builds again.
template <typename VT>
static void build_graph_any(Solve& S, Lane* lane) {
  try {
    build_graph<VT>(S, &lane->graph, &lane->graph_outer, &lane->graph_inner);
  } catch (const CudaError&) {
    if (!pdl_flag()) throw;
    cudaGetLastError();
    pdl_flag() = 0;
    build_graph<VT>(S, &lane->graph, &lane->graph_outer, &lane->graph_inner);
  }
}

template <typename VT>
static void setup_levels(Solve& S) {
  if (S.op->csr) {
    const CsrDev& C = S.op->cd;
    PROF(-1, -1, 0, 0, launch_csr_dinv<VT>(S.n, C.dk, C.dm, S.taus, S.n_tau, (cx<VT>*)S.dinv, S.s));
    CK(cudaMemsetAsync(S.singular, 0, sizeof(int), S.s));
    CK(cudaMemsetAsync(S.counter, 0, sizeof(int), S.s));
    S.lane->prof.all_launches += 2;
    return;
  }
  const auto& Ls = cycle_levels(S);
  const int bf = bf16_of(S) ? 1 : 0;
  {
    std::lock_guard<std::mutex> build_lock(g_build_mu);
    tail_prepare<VT>(tail_launch_smem<VT>(Ls, tail_level<VT>(Ls, tail_max_of<VT>(S.op))));
    fused_prepare<VT>();
    fused3d_prepare<VT>();
    size_t csm = 0;
    if (cluster_level<VT>(S.op, nullptr, &csm) >= 0) cluster_prepare<VT>(csm);
  }
  for (size_t l = 0; l < Ls.size(); ++l)
    PROF(-1, -1, 0, 0, launch_invd<VT>(Ls[l], S.taus, S.n_tau, (cx<VT>*)S.invd[l], S.s, bf));
  PROF(-1, -1, 0, 0, launch_diag64(Ls[0], S.taus, S.n_tau, S.diag64, S.s));
  if (S.tblob) {
    // the tail's coefficients per tau, laid out as in its shared memory
    const int lt = tail_level<VT>(Ls, tail_max_of<VT>(S.op));
    std::vector<int> cb;
    tail_layout<VT>(Ls, lt, true, &cb);
    for (int q = 0; q < S.n_tau; ++q)
      for (size_t l = lt; l < Ls.size(); ++l) {
        const LevelHost& L = Ls[l];
        unsigned char* dst = S.tblob + (size_t)q * S.tblob_bytes + (cb[l] - S.tcoef0);
        VT* const* src = sizeof(VT) == 8 ? (VT* const*)L.d64 : (VT* const*)L.d32;
        size_t nfx = face_count(L, 0), nfy = face_count(L, 1), nfz = L.nz > 1 ? face_count(L, 2) : 0;
        size_t off = 0;
        const size_t cnt[4] = {nfx, nfy, nfz, (size_t)L.n};
        for (int a = 0; a < 4; ++a) {
          if (cnt[a]) CK(cudaMemcpyAsync(dst + off, src[a], cnt[a] * sizeof(VT), cudaMemcpyDeviceToDevice, S.s));
          off += cnt[a] * sizeof(VT);
        }
        size_t realn = (nfx + nfy + nfz + L.n + 3) & ~(size_t)3;
        CK(cudaMemcpyAsync(dst + realn * sizeof(VT), (const cx<VT>*)S.invd[l] + (size_t)q * L.n,
                           sizeof(cx<VT>) * L.n, cudaMemcpyDeviceToDevice, S.s));
      }
  }
  const LevelHost& C = Ls.back();
  int64_t nc = C.n;
  CK(cudaMemsetAsync(S.singular, 0, sizeof(int), S.s));
  CK(cudaMemsetAsync(S.counter, 0, sizeof(int), S.s));
  CK(cudaMemsetAsync(S.bcount, 0, sizeof(int) * S.nslot, S.s));
  S.lane->prof.all_launches += 3;
  launch_coarse_inverse(C, S.taus, S.n_tau, S.cwork, S.cinv64, S.singular, S.s, bf);
  if constexpr (sizeof(VT) == 8) {
    CK(cudaMemcpyAsync(S.cinv, S.cinv64, sizeof(z64) * S.n_tau * nc * nc, cudaMemcpyDeviceToDevice, S.s));
  } else {
    PROF(-1, -1, 0, 0, launch_to_prec<VT>(S.cinv64, (cx<VT>*)S.cinv, (int64_t)S.n_tau * nc * nc, S.s));
  }
  ClusterParams<VT> CP{};
  const int lc = cluster_level<VT>(S.op, &CP);
  if (lc >= 0) {
    // the cluster kernel's band coefficients and coarsest inverse per tau
    std::vector<const cx<VT>*> iv(Ls.size());
    for (size_t l = 0; l < Ls.size(); ++l) iv[l] = (const cx<VT>*)S.invd[l];
    PROF(-1, -1, 0, 0, launch_cluster_blob<VT>(Ls, lc, CP, iv.data(), (const cx<VT>*)S.cinv, S.n_tau, S.cblob, S.s));
  }
}

template <typename VT>
static void carve(Solve& S, Arena& A, bool x_internal) {
  int64_t n = S.n;
  int ns = S.nslot, m = S.m, nf = S.n_f;
  auto& Ls = S.op->levels;
  A.reset();
  S.st = A.take<SlotState>(ns);
  S.b = A.take<z64>((size_t)ns * n);
  S.sigma = A.take<z64>(nf);
  S.taus = A.take<z64>(S.n_tau);
  S.sched = A.take<int32_t>(S.sched_len);
  S.rep_cyc = A.take<int32_t>((size_t)ns * m);
  S.rep_mj = A.take<int32_t>((size_t)ns * nf);
  S.V = A.take<z64>((size_t)ns * (m + 1) * n);
  // complex64 copy of the basis for the first CGS projection (mixed precision)
  S.V32 = S.precision != FKS_PREC_FP64 ? A.take<z32>((size_t)ns * (m + 1) * n) : nullptr;
  S.Z = A.take<z64>((size_t)ns * m * n);
  S.w = A.take<z64>((size_t)ns * n);
  S.ndef = defect_partials(S.op);
  if (S.op->csr) {
    S.f.assign(1, nullptr);
    S.z.clear();
    S.z2.clear();
    S.invd.clear();
    S.f[0] = A.take<cx<VT>>((size_t)ns * n);
    for (int i = 0; i < 9; ++i) S.bv[i] = A.take<cx<VT>>((size_t)ns * n);
    S.dinv = A.take<cx<VT>>((size_t)S.n_tau * n);
    if (S.amg) {
      const auto& sz = S.op->amg.sizes;
      S.amg_tab = A.take<AmgLevel<VT>>((size_t)S.n_tau * S.amg_L);
      for (int l = 0; l < S.amg_L; ++l) {
        S.amg_f[l] = l ? A.take<cx<VT>>((size_t)ns * sz[l]) : nullptr;
        S.amg_x[l] = A.take<cx<VT>>((size_t)ns * sz[l]);
        S.amg_y[l] = A.take<cx<VT>>((size_t)ns * sz[l]);
        S.amg_r[l] = A.take<cx<VT>>((size_t)ns * sz[l]);
      }
    }
    S.bsc = A.take<BcgScal>(ns);
    S.bpart = A.take<double>((size_t)ns * csr_blocks(n) * 3);
    S.cwork = S.cinv64 = nullptr;
    S.cinv = nullptr;
  } else {
    S.f.assign(Ls.size(), nullptr);
    S.z.assign(Ls.size(), nullptr);
    S.z2.assign(Ls.size(), nullptr);
    S.invd.assign(Ls.size(), nullptr);
    for (size_t l = 0; l < Ls.size(); ++l) {
      S.f[l] = A.take<cx<VT>>((size_t)ns * Ls[l].n);
      S.z[l] = A.take<cx<VT>>((size_t)ns * Ls[l].n);
      S.z2[l] = A.take<cx<VT>>((size_t)ns * Ls[l].n);
      S.invd[l] = A.take<cx<VT>>((size_t)S.n_tau * Ls[l].n);
    }
    S.diag64 = A.take<z64>((size_t)S.n_tau * n);
    S.tblob_bytes = tail_blob_bytes<VT>(Ls, tail_max_of<VT>(S.op), &S.tcoef0);
    S.tblob = S.tblob_bytes ? A.take<unsigned char>((size_t)S.n_tau * S.tblob_bytes) : nullptr;
    ClusterParams<VT> CP{};
    S.cblob = cluster_level<VT>(S.op, &CP) >= 0 ? A.take<unsigned char>((size_t)S.n_tau * CL_SIZE * CP.region)
                                                : nullptr;
    int64_t nc = Ls.back().n;
    S.cwork = A.take<z64>((size_t)S.n_tau * nc * nc);
    S.cinv64 = A.take<z64>((size_t)S.n_tau * nc * nc);
    S.cinv = A.take<cx<VT>>((size_t)S.n_tau * nc * nc);
  }
  S.singular = A.take<int32_t>(1);
  S.flags = A.take<int32_t>(ns);
  S.counter = A.take<int32_t>(1);
  S.bcount = A.take<int32_t>(ns);
  S.dpart = A.take<double>((size_t)ns * S.ndef * 2);
  S.npart = A.take<double>((size_t)ns * norm_blocks(n));
  S.mpart = A.take<double>((size_t)ns * norm_blocks(n));
  S.wpart = A.take<double>((size_t)ns * norm_blocks(n));
  S.mdpart = A.take<z64>((size_t)ns * mdot_blocks(n) * MAX_M);
  S.h12 = A.take<z64>((size_t)ns * 2 * MAX_M);
  S.H = A.take<z64>((size_t)ns * (m + 1) * m);
  S.taus_k = A.take<z64>((size_t)ns * m);
  S.pn = A.take<double>((size_t)ns * m);
  S.cyc = A.take<int32_t>((size_t)ns * m);
  S.g = A.take<z64>((size_t)ns * nf * (m + 1));
  S.rc = A.take<double>((size_t)ns * nf * m);
  S.rs = A.take<z64>((size_t)ns * nf * m);
  S.R = A.take<z64>((size_t)ns * nf * m * m);
  S.Y = A.take<z64>((size_t)ns * nf * m);
  S.sst = A.take<int32_t>((size_t)ns * nf);
  S.mj = A.take<int32_t>((size_t)ns * nf);
  S.est = A.take<double>((size_t)ns * nf);
  S.bnd = A.take<double>((size_t)ns * nf);
  S.alpha = A.take<double>((size_t)ns * nf);
  S.tolv = A.take<double>((size_t)ns * nf);
  S.rcoef = A.take<z64>((size_t)ns * nf);
  S.tpart = A.take<double>((size_t)ns * nf * (S.op->csr ? csr_blocks(n) : tres_blocks(Ls[0])));
  S.tres = A.take<double>((size_t)ns * nf);
  S.X = x_internal ? A.take<z64>((size_t)ns * nf * n) : nullptr;
  S.budget = S.batching ? A.take<int32_t>(1) : nullptr;
  S.stopv = S.batching ? A.take<int32_t>(ns) : nullptr;
  S.tcerr = S.batching ? A.take<int32_t>(1) : nullptr;
}

// Outputs of a run of consecutive slots [r0, r0 + nr) that belong to one
// caller (the server merges several requests into one batch); host or device.
struct OutGroup {
  int r0, nr;
  fks_c128* X;
  double *est, *bnd, *tru;
  int32_t *mj, *sst;
};

template <typename VT>
static fks_status solve_impl(fks_op* op, Lane* lane, const fks_c128* b, int n_rhs, const fks_c128* sigma, int n_f,
                             const fks_c128* tau, int n_tau, const fks_options* o, fks_c128* X, double* res_est,
                             double* res_bound, double* res_true, int32_t* m_j, int32_t* shift_status, fks_info* info,
                             cudaStream_t s, const std::vector<OutGroup>* groups = nullptr,
                             std::unique_lock<std::mutex>* api_lock = nullptr, const RestartIO* rio = nullptr) {
  Solve S{};
  S.op = op;
  S.lane = lane;
  S.s = s;
  S.api_lock = api_lock;
  S.nslot = n_rhs;
  S.n_f = n_f;
  S.n_tau = n_tau;
  S.m = o->m_max;
  S.sched_len = o->sched_len;
  S.precision = o->precision;
  S.variant = o->variant;
  S.n = op->n;
  S.tol = o->tol;
  S.eps = o->inner_tol > 0 ? o->inner_tol : std::min(1e-6, o->tol / 100.0);
  S.max_cycles = o->inner_max_cycles > 0 ? o->inner_max_cycles : 50;
  S.replay = o->replay_mode != 0;
  S.tolv_on = rio != nullptr;
  S.inner_steps = o->inner_steps > 0 ? o->inner_steps : (op->csr && op->amg.on ? 4 : 8);
  S.relax = o->inner_relax > 0 ? o->inner_relax : 0.0;
  {
    std::string err = amg_prepare<VT>(S, tau);
    if (!err.empty()) {
      set_error("fks_solve: " + err);
      return FKS_ERR_ARG;
    }
  }
  bool x_dev = groups ? false : is_device_ptr(X);
  if (groups && !res_true) res_true = (double*)1;  // grouped runs always compute true residuals
  // workspace size: carve once on a null base to measure
  Arena probe;
  carve<VT>(S, probe, !x_dev);
  size_t need = probe.off + 4096;
  lane->ws.reserve(need);
  carve<VT>(S, lane->ws, !x_dev);
  if (S.amg)
    CK(cudaMemcpyAsync(S.amg_tab, S.amg_table.data(), S.amg_table.size(), cudaMemcpyHostToDevice, s));
  z64* Xd = x_dev ? (z64*)X : S.X;
  bool x_early = false;  // host x_j already being copied on the lane's side stream
  std::vector<SlotState> st_host(n_rhs);
  S.st_host = st_host.data();
  int64_t n = S.n;
  int m = S.m;
  // inputs
  copy_in(S.b, b, sizeof(z64) * n * n_rhs, s);
  if (rio) CK(cudaMemcpyAsync(S.tolv, rio->tol_shift, sizeof(double) * n_f * n_rhs, cudaMemcpyHostToDevice, s));
  copy_in(S.sigma, sigma, sizeof(z64) * n_f, s);
  copy_in(S.taus, tau, sizeof(z64) * n_tau, s);
  CK(cudaMemcpyAsync(S.sched, o->tau_schedule, sizeof(int32_t) * o->sched_len, cudaMemcpyHostToDevice, s));
  if (S.replay) {
    CK(cudaMemcpyAsync(S.rep_cyc, o->replay_inner_cycles, sizeof(int32_t) * m * n_rhs, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(S.rep_mj, o->replay_mj, sizeof(int32_t) * n_f * n_rhs, cudaMemcpyHostToDevice, s));
  }
  // preconditioner setup for the distinct taus (inverse diagonals, coarse inverse)
  if (rio && rio->reuse_setup) {
    // a later restart cycle with the same layout: only the deciding kernels' counters
    CK(cudaMemsetAsync(S.counter, 0, sizeof(int), s));
    if (!op->csr) CK(cudaMemsetAsync(S.bcount, 0, sizeof(int) * S.nslot, s));
  } else {
    setup_levels<VT>(S);
  }
  // start: beta, v_1
  int nbn = norm_blocks(n);
  PROF(-1, -1, 0, 0, launch_norm2_partial(S.st, 0, S.b, n, n, S.npart, n_rhs, s));
  PROF(-1, -1, 0, 0, launch_start(S.st, n_rhs, S.npart, nbn, n_f, s));
  PROF(-1, -1, 0, 0, launch_init_v1(S.st, S.b, n, S.V, (m + 1) * n, n_rhs, s, S.V32));
  PROF(-1, -1, 0, 0, launch_init_shifts(S.st, n_f, m, S.sst, S.mj, S.est, S.bnd, S.Y, S.alpha, n_rhs, s));
  CK(cudaMemsetAsync(S.pn, 0, sizeof(double) * m * n_rhs, s));
  CK(cudaMemsetAsync(S.cyc, 0, sizeof(int32_t) * m * n_rhs, s));
  CK(cudaMemsetAsync(S.H, 0, sizeof(z64) * (m + 1) * m * n_rhs, s));
  CK(cudaMemsetAsync(S.taus_k, 0, sizeof(z64) * m * n_rhs, s));
  const int64_t vsV = (int64_t)(m + 1) * n, vsZ = (int64_t)m * n;
  int steps = 0;
  bool use_graph = o->launch_mode == 0;
  std::vector<int32_t> cyc_all((size_t)m * n_rhs);
  if (any_active(S)) {
    if (use_graph) {
      std::vector<double> key = {(double)(uintptr_t)lane->ws.base, (double)n_rhs, (double)n_f, (double)n_tau, (double)m,
                                 (double)S.sched_len, (double)S.precision, (double)S.variant, (double)S.replay,
                                 S.eps, S.tol, (double)S.max_cycles, (double)op->fuse_max[0],
                                 (double)op->fuse_max[1], (double)S.inner_steps, (double)op->tile16_max[0],
                                 (double)op->tile16_max[1], S.relax, (double)op->tail_max[0],
                                 (double)op->tail_max[1], (double)op->cluster_max[0], (double)op->cluster_max[1],
                                 (double)op->tile8_max[0], (double)op->tile8_max[1], (double)S.tolv_on,
                                 (double)(S.amg ? op->amg.gen : -1), (double)S.amg_L, (double)S.batching};
      for (int pz = 0; pz < 2; ++pz)
        for (int l = 0; l < MAX_LEVELS; ++l) key.push_back((double)op->zchunk[pz][l]);
      key.push_back((double)op->coop_max[0]);
      key.push_back((double)op->coop_max[1]);
      key.push_back((double)pdl_flag());
      if (!lane->graph || lane->graph_key != key) {
        if (lane->graph) cudaGraphExecDestroy(lane->graph);
        lane->graph = nullptr;
        build_graph_any<VT>(S, lane);
        key.back() = (double)pdl_flag();
        lane->graph_key = key;
      }
      CK(cudaGraphLaunch(lane->graph, s));
      if (S.api_lock) {
        // let other batches set up and launch while this graph runs
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, s));
        S.api_lock->unlock();
        cudaError_t we = cudaEventSynchronize(ev);
        S.api_lock->lock();
        cudaEventDestroy(ev);
        CK(we);
      }
      // launch count: per step the outer section, per inner iteration the inner section
      CK(cudaMemcpyAsync(cyc_all.data(), S.cyc, sizeof(int32_t) * m * n_rhs, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(S.st_host, S.st, sizeof(SlotState) * n_rhs, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int r = 0; r < n_rhs; ++r) steps = std::max(steps, S.st_host[r].k);
      int64_t inner_iters = 0;
      for (int k = 0; k < steps; ++k) {
        int mx = 0;
        for (int r = 0; r < n_rhs; ++r) mx = std::max(mx, cyc_all[(size_t)r * m + k]);
        inner_iters += mx;
      }
      lane->prof.all_launches += (int64_t)steps * lane->graph_outer + inner_iters * lane->graph_inner;
    } else {
      for (int step = 1; step <= m; ++step) {
        steps = step;
        sec_step_begin(S);
        inner_solve<VT>(S, S.V, vsV, S.Z, vsZ);
        sec_step_end(S, step, 0, 0);
        if (!any_active(S)) break;
      }
    }
  }
  // assembly and true residual
  int tc_err_h = 0;
  int* tc_err = nullptr;
  {
    const double ns = n_rhs, nn = (double)n, ks = steps, d = op->dim;
    // each source's own step count decides its kernel, so that a source is
    // assembled the same way alone and in a batch
    CK(cudaMemcpyAsync(S.st_host, S.st, sizeof(SlotState) * n_rhs, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int k_tc = 0;
    bool any_fp64 = false;
    for (int r = 0; r < n_rhs; ++r) {
      if (tc_supported(std::max(S.st_host[r].k, 1), n)) k_tc = std::max(k_tc, S.st_host[r].k);
      else any_fp64 = true;
    }
    const bool use_tc = o->assembly == 0 && k_tc >= 1;
    if (use_tc) {
      // tensor cores: slices of Z and Y, the product, the epilogue; sources in
      // groups of tc_group_size, whose slices the workspace holds at a time
      const int sb = tc_group_size(n, n_f, k_tc, n_rhs);
      TcLayout T = tc_layout(n, n_f, k_tc, sb);
      const size_t need = tc_ws_bytes(T);
      lane->tcws.reserve(need + 256);
      tc_err = (int*)(lane->tcws.base + need);
      {
        std::lock_guard<std::mutex> build_lock(g_build_mu);
        tc_prepare();
      }
      CK(cudaMemsetAsync(tc_err, 0, sizeof(int), s));
      lane->prof.all_launches += 1;
      for (int r0 = 0; r0 < n_rhs; r0 += sb) {
        const int nr = std::min(sb, n_rhs - r0);
        const double kt = k_tc, kp = 16.0 * T.nslab, nsb = nr;
        int launched = 0;
        PROF(FKS_K_ASSEMBLE, -1, nsb * (2 * 16 * nn * kt + 2 * 16 * nn * kp + 16 * nn * n_f),
             nsb * 8 * nn * kt * n_f,
             launched = launch_tc_assemble(T, S.st + r0, S.Z + (size_t)r0 * vsZ, vsZ, S.Y + (size_t)r0 * n_f * m,
                                           S.mj + (size_t)r0 * n_f, n_f, m, Xd + (size_t)r0 * n_f * n, n, nr,
                                           lane->tcws.base, tc_err, s));
        lane->prof.all_launches += launched - 1;  // the two slicing kernels beyond the one PROF counted
      }
    }
    if (!use_tc || any_fp64) {
      const int skip = use_tc ? TC_MAX_KP / 2 : -1;  // sources up to this step count were done above
      PROF(FKS_K_ASSEMBLE, -1, ns * 16 * nn * (ks + n_f), ns * 8 * nn * ks * n_f,
           launch_assemble(S.Z, vsZ, S.Y, S.mj, n_f, m, Xd, n, n_rhs, s, use_tc ? S.st : nullptr, skip));
    }
    if (!groups && !x_dev && X && res_true) {
      // host x_j: copy them on the side stream while the true residuals run
      lane->side_init();
      CK(cudaEventRecord(lane->ev_x, s));
      CK(cudaStreamWaitEvent(lane->side, lane->ev_x, 0));
      copy_out(X, Xd, sizeof(z64) * n * n_f * n_rhs, lane->side);
      CK(cudaEventRecord(lane->ev_copied, lane->side));
      x_early = true;
    }
    if (res_true && op->csr)
      PROF(FKS_K_TRES, -1, ns * (nn * (16.0 * n_f + 16) + n_f * op->cd.nnz * 36.0), ns * n_f * op->cd.nnz * 10.0,
           launch_csr_true_residual(op->cd.view<double>(n), S.sigma, n_f, S.b, Xd, S.tpart, S.st, S.tres, n_rhs, s));
    else if (res_true)
      PROF(FKS_K_TRES, -1, ns * nn * (16.0 * n_f + 16 + 8 * (d + 1)), ns * nn * n_f * (8 * d + 14),
           launch_true_residual(op->levels[0], S.sigma, n_f, S.b, Xd, S.tpart, S.st, S.tres, n_rhs, s));
    if (res_true) lane->prof.all_launches += 1;  // the true residual is two kernels
  }
  CK(cudaGetLastError());
  // outputs
  std::vector<int32_t> sst_h((size_t)n_f * n_rhs);
  CK(cudaMemcpyAsync(sst_h.data(), S.sst, sizeof(int32_t) * n_f * n_rhs, cudaMemcpyDeviceToHost, s));
  if (groups) {
    for (const OutGroup& g : *groups) {
      size_t o0 = (size_t)g.r0 * n_f, cnt = (size_t)g.nr * n_f;
      copy_out(g.X, Xd + o0 * n, sizeof(z64) * n * cnt, s);
      copy_out(g.est, S.est + o0, sizeof(double) * cnt, s);
      copy_out(g.bnd, S.bnd + o0, sizeof(double) * cnt, s);
      copy_out(g.tru, S.tres + o0, sizeof(double) * cnt, s);
      copy_out(g.mj, S.mj + o0, sizeof(int32_t) * cnt, s);
      copy_out(g.sst, S.sst + o0, sizeof(int32_t) * cnt, s);
    }
  } else {
    if (!x_dev && !x_early) copy_out(X, Xd, sizeof(z64) * n * n_f * n_rhs, s);
    if (x_early) CK(cudaStreamWaitEvent(s, lane->ev_copied, 0));
    copy_out(res_est, S.est, sizeof(double) * n_f * n_rhs, s);
    copy_out(res_bound, S.bnd, sizeof(double) * n_f * n_rhs, s);
    if (res_true) copy_out(res_true, S.tres, sizeof(double) * n_f * n_rhs, s);
    copy_out(m_j, S.mj, sizeof(int32_t) * n_f * n_rhs, s);
    copy_out(shift_status, S.sst, sizeof(int32_t) * n_f * n_rhs, s);
  }
  std::vector<int32_t> cyc_h;
  std::vector<double> pn_h;
  if (info && info->inner_cycles) cyc_h.resize((size_t)m * n_rhs);
  if (info && info->pnorm) pn_h.resize((size_t)m * n_rhs);
  if (!cyc_h.empty()) CK(cudaMemcpyAsync(cyc_h.data(), S.cyc, sizeof(int32_t) * m * n_rhs, cudaMemcpyDeviceToHost, s));
  if (info && info->gmres_alpha) copy_out(info->gmres_alpha, S.alpha, sizeof(double) * n_f * n_rhs, s);
  if (info && info->hbar) copy_out(info->hbar, S.H, sizeof(z64) * (m + 1) * m * n_rhs, s);
  if (info && info->tau_k) copy_out(info->tau_k, S.taus_k, sizeof(z64) * m * n_rhs, s);
  if (rio) CK(cudaMemcpyAsync(rio->coef, S.rcoef, sizeof(z64) * n_f * n_rhs, cudaMemcpyDeviceToHost, s));
  if (!pn_h.empty()) CK(cudaMemcpyAsync(pn_h.data(), S.pn, sizeof(double) * m * n_rhs, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(S.st_host, S.st, sizeof(SlotState) * n_rhs, cudaMemcpyDeviceToHost, s));
  int singular = 0;
  CK(cudaMemcpyAsync(&singular, S.singular, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (tc_err) CK(cudaMemcpyAsync(&tc_err_h, tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  if (info) {
    for (int r = 0; r < n_rhs; ++r) {
      if (info->steps) info->steps[r] = S.st_host[r].beta > 0 ? S.st_host[r].k : 0;
      if (info->breakdown) info->breakdown[r] = S.st_host[r].breakdown;
    }
    if (info->inner_cycles) std::memcpy(info->inner_cycles, cyc_h.data(), sizeof(int32_t) * m * n_rhs);
    if (info->pnorm) std::memcpy(info->pnorm, pn_h.data(), sizeof(double) * m * n_rhs);
  }
  (void)steps;
  if (rio) {
    // the common residual direction v_{k+1} of each source for the next cycle
    for (int r = 0; r < n_rhs; ++r) {
      rio->beta[r] = S.st_host[r].beta;
      rio->steps[r] = S.st_host[r].beta > 0 ? S.st_host[r].k : 0;
      if (rio->steps[r] > 0)
        CK(cudaMemcpyAsync(rio->v_next + (size_t)r * n, S.V + (size_t)r * (m + 1) * n + (size_t)rio->steps[r] * n,
                           sizeof(z64) * n, cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaStreamSynchronize(s));
  }
  if (tc_err_h) {
    set_error("tensor-core assembly: a wait for copies or MMAs gave up after two seconds");
    return FKS_ERR_CUDA;
  }
  if (singular) {
    set_error("coarsest multigrid level is singular for some tau");
    return FKS_ERR_ARG;
  }
  bool nc = false, bd = false, capped = false;
  for (int32_t v : sst_h) {
    if (v == 1 || v == -1) nc = true;
    if (v == 2) bd = true;
  }
  for (int r = 0; r < n_rhs; ++r) capped = capped || S.st_host[r].inner_capped;
  if (nc) return FKS_NOT_CONVERGED;
  if (bd) return FKS_BREAKDOWN_EXACT;
  if (capped) return FKS_INNER_NOT_CONVERGED;
  return FKS_OK;
}

static bool finite_c(const fks_c128& z) { return std::isfinite(z.re) && std::isfinite(z.im); }

static int status_rank(fks_status s) {
  switch (s) {
    case FKS_NOT_CONVERGED: return 3;
    case FKS_BREAKDOWN_EXACT: return 2;
    case FKS_INNER_NOT_CONVERGED: return 1;
    default: return 0;
  }
}

// Sources are solved in lockstep batches sized to the free device memory:
// one batch when they all fit, otherwise equal batches one after another.
// Restarted flexible FOM (Section 2.2.2): FOM residuals of all shifts are
// collinear, r_j = c_j v_{k+1} (Eq. fomresidualsimplified), so a cycle of at
// most restart_len steps is followed by one on v_{k+1} for the shifts not yet
// certified, each with its right-hand side scaled by its own coefficient.
// With the residual estimate C_j v of the current iterate and the part A_j that
// the estimates of the finished cycles did not see (Eq. trueresidual), shift j
// is certified when its cycle's bound reaches (tol ||b|| - A_j) / |C_j| (its
// per-shift tolerance), and x_j += C_j d_j. The tau schedule continues across
// cycles. One source at a time; every cycle is an ordinary solve_impl.
template <typename VT>
static fks_status solve_restarted(fks_op* op, Lane* lane, const fks_c128* b, int n_rhs, const fks_c128* sigma,
                                  int n_f, const fks_c128* tau, int n_tau, const fks_options* o, fks_c128* X,
                                  double* res_est, double* res_bound, double* res_true, int32_t* m_j,
                                  int32_t* shift_status, fks_info* info, cudaStream_t s) {
  const int64_t n = op->n;
  const int len = o->restart_len;
  const int max_cycles = (o->max_restarts > 0 ? o->max_restarts : 20) + 1;
  const double tol = o->tol;
  std::vector<fks_c128> sg(n_f);
  CK(cudaMemcpy(sg.data(), sigma, sizeof(fks_c128) * n_f, cudaMemcpyDefault));
  const int nblk = op->csr ? csr_blocks(n) : tres_blocks(op->levels[0]);
  // device buffers of one source: accumulated x, a cycle's x, residual directions,
  // right-hand side, and the final true residual's inputs
  std::vector<void*> owned;
  auto dmalloc = [&](size_t bytes) {
    void* p = nullptr;
    CK(cudaMallocAsync(&p, bytes, s));
    owned.push_back(p);
    return p;
  };
  struct Freer {
    std::vector<void*>& v;
    cudaStream_t s;
    ~Freer() { for (void* p : v) cudaFreeAsync(p, s); }
  } freer{owned, s};
  z64* xacc = (z64*)dmalloc(sizeof(z64) * n * n_f);
  z64* xhat = (z64*)dmalloc(sizeof(z64) * n * n_f);
  z64* vcur = (z64*)dmalloc(sizeof(z64) * n);
  z64* vnext = (z64*)dmalloc(sizeof(z64) * n);
  z64* bdev = (z64*)dmalloc(sizeof(z64) * n);
  z64* sgd = (z64*)dmalloc(sizeof(z64) * n_f);
  double* tpart = (double*)dmalloc(sizeof(double) * n_f * nblk);
  double* trd = (double*)dmalloc(sizeof(double) * n_f);
  SlotState* std_ = (SlotState*)dmalloc(sizeof(SlotState));
  int32_t* idxd = (int32_t*)dmalloc(sizeof(int32_t) * n_f);
  z64* acd = (z64*)dmalloc(sizeof(z64) * n_f);
  CK(cudaMemcpyAsync(sgd, sg.data(), sizeof(z64) * n_f, cudaMemcpyHostToDevice, s));
  std::vector<double> est((size_t)n_f * n_rhs), bnd((size_t)n_f * n_rhs), tru((size_t)n_f * n_rhs);
  std::vector<int32_t> mj((size_t)n_f * n_rhs), sst((size_t)n_f * n_rhs);
  bool any_nc = false, any_bd = false;
  for (int r = 0; r < n_rhs; ++r) {
    CK(cudaMemsetAsync(xacc, 0, sizeof(z64) * n * n_f, s));
    copy_in(bdev, b + (size_t)r * n, sizeof(z64) * n, s);
    std::vector<std::complex<double>> C(n_f, 1.0);
    std::vector<double> A(n_f, 0.0);
    std::vector<int> live(n_f);
    for (int j = 0; j < n_f; ++j) live[j] = j;
    double beta0 = 0.0;
    int done_steps = 0;
    bool breakdown = false;
    double* er = est.data() + (size_t)r * n_f;
    double* br = bnd.data() + (size_t)r * n_f;
    int32_t* mr = mj.data() + (size_t)r * n_f;
    int32_t* sr = sst.data() + (size_t)r * n_f;
    for (int j = 0; j < n_f; ++j) sr[j] = FKS_NOT_CONVERGED;
    // Every cycle passes all shifts, those already certified (or abandoned) with an
    // infinite tolerance (they freeze at the first step and are ignored), so the
    // workspace layout, the preconditioner setup and the captured graph of the
    // first cycle serve every later one.
    std::vector<double> tl(n_f);
    std::vector<double> e_c(n_f), b_c(n_f);
    std::vector<int32_t> m_c(n_f), s_c(n_f);
    std::vector<z64> coef(n_f);
    std::vector<int32_t> sched(o->sched_len);
    const double inf = std::numeric_limits<double>::infinity();
    for (int cyc = 0; cyc < max_cycles && !live.empty(); ++cyc) {
      std::fill(tl.begin(), tl.end(), inf);
      std::vector<int> nlive;
      for (int j : live) {
        // cycle 0 solves with b itself (figures relative to ||b||), later ones with a unit v
        const double t = cyc == 0 ? tol : (tol * beta0 - A[j]) / std::abs(C[j]);
        if (t > 0.0) {   // otherwise the carried error alone exceeds the tolerance: not certifiable
          tl[j] = t;
          nlive.push_back(j);
        }
      }
      live = nlive;
      if (live.empty()) break;
      for (int i = 0; i < o->sched_len; ++i) sched[i] = o->tau_schedule[(done_steps + i) % o->sched_len];
      fks_options oc = *o;
      oc.m_max = len;
      oc.tau_schedule = sched.data();
      oc.restart_len = 0;
      // the relaxed inner tolerance of a cycle follows its shifts' own tolerances
      // (relative to its unit right-hand side), not the original one
      oc.tol = inf;
      for (int j : live) oc.tol = std::min(oc.tol, tl[j]);
      double beta_c = 0.0;
      int32_t steps_c = 0;
      RestartIO rio{tl.data(), coef.data(), &beta_c, &steps_c, vnext, cyc > 0 ? 1 : 0};
      const fks_c128* rhs = cyc == 0 ? (const fks_c128*)bdev : (const fks_c128*)vcur;
      fks_status st = solve_impl<VT>(op, lane, rhs, 1, sg.data(), n_f, tau, n_tau, &oc, (fks_c128*)xhat, e_c.data(),
                                     b_c.data(), nullptr, m_c.data(), s_c.data(), nullptr, s, nullptr, nullptr, &rio);
      if (st < 0) return st;
      if (cyc == 0) {
        beta0 = beta_c;
        if (beta0 == 0.0) {   // zero right-hand side: x = 0 for every shift
          for (int j = 0; j < n_f; ++j) { sr[j] = FKS_OK; er[j] = br[j] = 0.0; mr[j] = 0; }
          live.clear();
          break;
        }
      }
      // x_j += a_j d_j with a_j = 1 on the first cycle (its right-hand side is b), C_j after
      const int nk = (int)live.size();
      std::vector<int32_t> idx(nk);
      std::vector<z64> acoef(nk);
      for (int i = 0; i < nk; ++i) {
        idx[i] = live[i];
        const std::complex<double> a = cyc == 0 ? std::complex<double>(1.0) : C[live[i]];
        acoef[i] = mk(a.real(), a.imag());
      }
      CK(cudaMemcpyAsync(idxd, idx.data(), sizeof(int32_t) * nk, cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(acd, acoef.data(), sizeof(z64) * nk, cudaMemcpyHostToDevice, s));
      launch_axpy_cols(xacc, xhat, idxd, acd, nk, n, s);
      CK(cudaGetLastError());
      std::vector<int> next;
      for (int i = 0; i < nk; ++i) {
        const int j = live[i];
        const double sc = cyc == 0 ? beta0 : std::abs(C[j]);   // absolute scale of the cycle's relative figures
        const double rs = cyc == 0 ? 1.0 : sc / beta0;         // the same, relative to ||b||
        const std::complex<double> a(acoef[i].re, acoef[i].im);
        if (s_c[j] == FKS_OK || s_c[j] == FKS_BREAKDOWN_EXACT) {
          sr[j] = s_c[j];
          er[j] = rs * e_c[j];
          br[j] = rs * b_c[j] + A[j] / beta0;
          mr[j] = done_steps + m_c[j];
        } else {
          A[j] += sc * (b_c[j] - e_c[j]);
          C[j] = a * std::complex<double>(coef[j].re, coef[j].im);
          er[j] = std::abs(C[j]) / beta0;
          br[j] = (std::abs(C[j]) + A[j]) / beta0;
          mr[j] = done_steps + m_c[j];
          next.push_back(j);
        }
      }
      done_steps += steps_c;
      if (steps_c < len && !next.empty()) breakdown = true;  // cannot happen without a breakdown status
      live = next;
      std::swap(vcur, vnext);
      if (breakdown) break;
    }
    for (int j = 0; j < n_f; ++j) {
      if (sr[j] == FKS_NOT_CONVERGED) any_nc = true;
      if (sr[j] == FKS_BREAKDOWN_EXACT) any_bd = true;
    }
    // true residuals of the accumulated x against b
    if (res_true) {
      SlotState sh{};
      sh.beta = beta0;
      CK(cudaMemcpyAsync(std_, &sh, sizeof(SlotState), cudaMemcpyHostToDevice, s));
      if (op->csr)
        launch_csr_true_residual(op->cd.view<double>(n), sgd, n_f, bdev, xacc, tpart, std_, trd, 1, s);
      else
        launch_true_residual(op->levels[0], sgd, n_f, bdev, xacc, tpart, std_, trd, 1, s);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(tru.data() + (size_t)r * n_f, trd, sizeof(double) * n_f, cudaMemcpyDeviceToHost, s));
    }
    copy_out(X + (size_t)r * n_f * n, xacc, sizeof(z64) * n * n_f, s);
    CK(cudaStreamSynchronize(s));
    if (info) {
      if (info->steps) info->steps[r] = done_steps;
      if (info->breakdown) info->breakdown[r] = breakdown ? 1 : 0;
    }
  }
  copy_out(res_est, est.data(), sizeof(double) * n_f * n_rhs, s);
  copy_out(res_bound, bnd.data(), sizeof(double) * n_f * n_rhs, s);
  if (res_true) copy_out(res_true, tru.data(), sizeof(double) * n_f * n_rhs, s);
  copy_out(m_j, mj.data(), sizeof(int32_t) * n_f * n_rhs, s);
  copy_out(shift_status, sst.data(), sizeof(int32_t) * n_f * n_rhs, s);
  CK(cudaStreamSynchronize(s));
  return any_nc ? FKS_NOT_CONVERGED : (any_bd ? FKS_BREAKDOWN_EXACT : FKS_OK);
}

template <typename VT>
static fks_status solve_chunked(fks_op* op, Lane* lane, const fks_c128* b, int n_rhs, const fks_c128* sigma, int n_f,
                                const fks_c128* tau, int n_tau, const fks_options* o, fks_c128* X, double* res_est,
                                double* res_bound, double* res_true, int32_t* m_j, int32_t* shift_status,
                                fks_info* info, cudaStream_t s) {
  bool x_dev = is_device_ptr(X);
  auto ws_bytes = [&](int ns) {
    Solve S{};
    S.op = op;
    S.nslot = ns;
    S.n_f = n_f;
    S.n_tau = n_tau;
    S.m = o->m_max;
    S.sched_len = o->sched_len;
    S.precision = o->precision;
    S.n = op->n;
    Arena probe;
    carve<VT>(S, probe, !x_dev);
    // the tensor-core assembly's slices of the first group of sources
    const int kmax = std::min(o->m_max, TC_MAX_KP / 2);
    const size_t tc = o->assembly == 0 && tc_supported(kmax, op->n)
                          ? tc_ws_bytes(tc_layout(op->n, n_f, kmax, tc_group_size(op->n, n_f, kmax, ns)))
                          : 0;
    return probe.off + tc + 4096;
  };
  size_t one = ws_bytes(1), two = ws_bytes(2);
  size_t per = two > one ? two - one : one, fixed = one > per ? one - per : 0;
  size_t freeb = 0, totb = 0;
  CK(cudaMemGetInfo(&freeb, &totb));
  size_t avail = freeb + lane->ws.cap;
  size_t reserve = std::min<size_t>(avail / 20, size_t(2) << 30);
  avail = avail > reserve ? avail - reserve : 0;
  int max_slots = (int)std::max<size_t>(1, avail > fixed ? (avail - fixed) / per : 1);
  int nchunk = (n_rhs + max_slots - 1) / max_slots;
  int chunk = (n_rhs + nchunk - 1) / nchunk;
  if (nchunk == 1)
    return solve_impl<VT>(op, lane, b, n_rhs, sigma, n_f, tau, n_tau, o, X, res_est, res_bound, res_true, m_j,
                          shift_status, info, s);
  fks_status worst = FKS_OK;
  for (int r0 = 0; r0 < n_rhs; r0 += chunk) {
    int nr = std::min(chunk, n_rhs - r0);
    fks_options oc = *o;
    if (o->replay_mode) {
      oc.replay_inner_cycles = o->replay_inner_cycles + (size_t)r0 * o->m_max;
      oc.replay_mj = o->replay_mj + (size_t)r0 * n_f;
    }
    fks_info ic{};
    if (info) {
      ic.steps = info->steps ? info->steps + r0 : nullptr;
      ic.inner_cycles = info->inner_cycles ? info->inner_cycles + (size_t)r0 * o->m_max : nullptr;
      ic.pnorm = info->pnorm ? info->pnorm + (size_t)r0 * o->m_max : nullptr;
      ic.breakdown = info->breakdown ? info->breakdown + r0 : nullptr;
      ic.gmres_alpha = info->gmres_alpha ? info->gmres_alpha + (size_t)r0 * n_f : nullptr;
      ic.hbar = info->hbar ? info->hbar + (size_t)r0 * (o->m_max + 1) * o->m_max : nullptr;
      ic.tau_k = info->tau_k ? info->tau_k + (size_t)r0 * o->m_max : nullptr;
    }
    size_t nf = (size_t)n_f * r0;
    fks_status st = solve_impl<VT>(op, lane, b + (size_t)r0 * op->n, nr, sigma, n_f, tau, n_tau, &oc,
                                   X + (size_t)r0 * n_f * op->n, res_est + nf, res_bound + nf,
                                   res_true ? res_true + nf : nullptr, m_j + nf, shift_status + nf,
                                   info ? &ic : nullptr, s);
    if (st < 0) return st;
    if (status_rank(st) > status_rank(worst)) worst = st;
  }
  return worst;
}

// A CSR operator's Jacobi preconditioner needs a nonzero diagonal of K + tau M.
static bool csr_diag_ok(const fks_op* op, const fks_c128* tau, int n_tau) {
  if (!op->csr) return true;
  for (int q = 0; q < n_tau; ++q)
    for (int64_t i = 0; i < op->n; ++i) {
      double re = op->cd.dk_h[i] + tau[q].re * op->cd.dm_h[i], im = tau[q].im * op->cd.dm_h[i];
      if (re == 0.0 && im == 0.0) return false;
    }
  return true;
}

}  // namespace fks

// ====================================================================== C ABI
extern "C" {

const char* fks_last_error(void) { return fks::get_error(); }
const char* fks_version(void) { return "fks 0.1 (sm_103a)"; }

fks_status fks_create(fks_ctx** out, int device) {
  if (!out) { set_error("fks_create: out is NULL"); return FKS_ERR_ARG; }
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
    cudaGetLastError();
    set_error("fks_create: no CUDA device");
    return FKS_ERR_CUDA;
  }
  if (device < 0 || device >= count) { set_error("fks_create: bad device index"); return FKS_ERR_ARG; }
  if (cudaSetDevice(device) != cudaSuccess) { set_error("fks_create: cudaSetDevice failed"); return FKS_ERR_CUDA; }
  fks_ctx* c = new fks_ctx;
  c->device = device;
  *out = c;
  set_error("");
  return FKS_OK;
}

void fks_destroy(fks_ctx* ctx) { delete ctx; }

fks_status fks_op_grid(fks_ctx* ctx, int dim, const int64_t ncell[3], const double h[3], const double* cond,
                       const double* ss, uint32_t mask, fks_op** out) {
  if (!out) { set_error("fks_op_grid: out is NULL"); return FKS_ERR_ARG; }
  *out = nullptr;
  if (!ctx || !ncell || !h || !cond || !ss) { set_error("fks_op_grid: NULL argument"); return FKS_ERR_ARG; }
  if (dim != 2 && dim != 3) { set_error("fks_op_grid: dim must be 2 or 3"); return FKS_ERR_ARG; }
  int64_t nx = ncell[0], ny = ncell[1], nz = dim == 3 ? ncell[2] : 1;
  if (nx < 1 || ny < 1 || nz < 1 || nx > (1 << 30) || ny > (1 << 30) || nz > (1 << 30)) {
    set_error("fks_op_grid: cell counts must be >= 1");
    return FKS_ERR_ARG;
  }
  for (int a = 0; a < dim; ++a)
    if (!(h[a] > 0) || !std::isfinite(h[a])) { set_error("fks_op_grid: h must be positive"); return FKS_ERR_ARG; }
  if (mask >> (2 * dim)) { set_error("fks_op_grid: dirichlet_mask has bits beyond 2*dim"); return FKS_ERR_ARG; }
  int64_t n = nx * ny * nz;
  for (int64_t c = 0; c < n; ++c) {
    if (!(cond[c] > 0) || !std::isfinite(cond[c])) { set_error("fks_op_grid: cond must be positive and finite"); return FKS_ERR_ARG; }
    if (!(ss[c] > 0) || !std::isfinite(ss[c])) { set_error("fks_op_grid: ss must be positive and finite"); return FKS_ERR_ARG; }
  }
  double hh[3] = {h[0], h[1], dim == 3 ? h[2] : 1.0};
  // lumped storage: M_cc = S_s,c * cell volume
  double vol = hh[0] * hh[1] * hh[2];
  std::vector<double> mass(n);
  for (int64_t c = 0; c < n; ++c) mass[c] = ss[c] * vol;
  std::vector<LevelHost> Ls = level_shapes((int)nx, (int)ny, (int)nz, hh, false);
  if (Ls.back().n > MAX_COARSE) Ls = level_shapes((int)nx, (int)ny, (int)nz, hh, true);
  if (Ls.back().n > MAX_COARSE) {
    set_error("fks_op_grid: coarsest multigrid level has more than 1024 cells (more than 16 levels needed)");
    return FKS_ERR_ARG;
  }
  fks_op* op = new fks_op;
  op->ctx = ctx;
  op->dim = dim;
  op->nx = (int)nx; op->ny = (int)ny; op->nz = (int)nz;
  op->n = n;
  op->mask = mask;
  double* cond_d = nullptr;
  try {
    CK(cudaSetDevice(ctx->device));
    for (auto& L : Ls) {
      for (int a = 0; a < 4; ++a) {
        int64_t cnt = a < 3 ? (a == 2 && L.nz == 1 ? 1 : face_count(L, a)) : L.n;
        CK(cudaMalloc(&L.d64[a], sizeof(double) * cnt));
        CK(cudaMalloc(&L.d32[a], sizeof(float) * cnt));
        CK(cudaMalloc(&L.d16[a], sizeof(__nv_bfloat16) * cnt));
        CK(cudaMalloc(&L.d32b[a], sizeof(float) * cnt));
      }
    }
    op->levels = Ls;
    cudaStream_t s = 0;
    CK(cudaMalloc(&cond_d, sizeof(double) * n));
    CK(cudaMemcpy(cond_d, cond, sizeof(double) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(op->levels[0].d64[3], mass.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    launch_faces_from_cond(op->levels[0], hh, mask, cond_d, s);
    {
      // coarse-face factors of every coarsening from the cells' widths (in
      // finest cells) along each axis, uploaded at once
      std::vector<double> w[3] = {std::vector<double>(nx, 1.0), std::vector<double>(ny, 1.0),
                                  std::vector<double>(nz, 1.0)};
      std::vector<double> all;
      std::vector<size_t> at;
      for (size_t l = 0; l + 1 < op->levels.size(); ++l) {
        const LevelHost& F = op->levels[l];
        const int r[3] = {F.rx, F.ry, F.rz};
        for (int a = 0; a < 3; ++a) {
          std::vector<double> W;
          std::vector<double> f = coarse_face_factors(w[a], r[a], &W);
          at.push_back(all.size());
          all.insert(all.end(), f.begin(), f.end());
          w[a] = W;
        }
      }
      double* fac_d = nullptr;
      if (!all.empty()) {
        CK(cudaMalloc(&fac_d, sizeof(double) * all.size()));
        CK(cudaMemcpy(fac_d, all.data(), sizeof(double) * all.size(), cudaMemcpyHostToDevice));
      }
      for (size_t l = 0; l + 1 < op->levels.size(); ++l)
        launch_coarsen(op->levels[l], op->levels[l + 1], fac_d + at[3 * l], fac_d + at[3 * l + 1],
                       fac_d + at[3 * l + 2], s);
      if (fac_d) {
        CK(cudaStreamSynchronize(s));
        CK(cudaFree(fac_d));
      }
    }
    CK(cudaMalloc(&op->levels[0].kd64, sizeof(double) * n));
    launch_kdiag(op->levels[0], op->levels[0].kd64, s);
    for (auto& L : op->levels)
      for (int a = 0; a < 4; ++a) {
        int64_t cnt = a < 3 ? (a == 2 && L.nz == 1 ? 1 : face_count(L, a)) : L.n;
        launch_to_f32(L.d64[a], L.d32[a], cnt, s);
        launch_round_bf16(L.d64[a], L.d16[a], L.d32b[a], cnt, s);
      }
    // the bf16-smoother option's view of the hierarchy: the kernels that read
    // fp32 coefficients get the bf16-rounded values, so every kernel of its
    // V-cycle works with the same coefficients
    op->levels_bf = op->levels;
    for (auto& L : op->levels_bf)
      for (int a = 0; a < 4; ++a) L.d32[a] = L.d32b[a];
    CK(cudaDeviceSynchronize());
    CK(cudaGetLastError());
    op->cond_d = cond_d;
  } catch (CudaError& e) {
    if (cond_d) cudaFree(cond_d);
    set_error(std::string("fks_op_grid: ") + e.where + ": " + cudaGetErrorString(e.e));
    fks_op_destroy(op);
    return e.e == cudaErrorMemoryAllocation ? FKS_ERR_OOM : FKS_ERR_CUDA;
  }
  *out = op;
  return FKS_OK;
}

fks_status fks_op_csr(fks_ctx* ctx, int64_t n, const int64_t* k_rowptr, const int32_t* k_col, const double* k_val,
                      const int64_t* m_rowptr, const int32_t* m_col, const double* m_val, fks_op** out) {
  if (!out) { set_error("fks_op_csr: out is NULL"); return FKS_ERR_ARG; }
  *out = nullptr;
  if (!ctx || !k_rowptr || !m_rowptr) { set_error("fks_op_csr: NULL argument"); return FKS_ERR_ARG; }
  if (n < 1 || n > INT32_MAX) { set_error("fks_op_csr: n must be in 1..2^31-1"); return FKS_ERR_ARG; }
  // checks of both matrices
  const int64_t* rp[2] = {k_rowptr, m_rowptr};
  const int32_t* cl[2] = {k_col, m_col};
  const double* vl[2] = {k_val, m_val};
  for (int a = 0; a < 2; ++a) {
    if (rp[a][0] != 0) { set_error("fks_op_csr: row pointers must start at 0"); return FKS_ERR_ARG; }
    for (int64_t i = 0; i < n; ++i)
      if (rp[a][i + 1] < rp[a][i]) { set_error("fks_op_csr: row pointers must not decrease"); return FKS_ERR_ARG; }
    int64_t nz = rp[a][n];
    if (nz > 0 && (!cl[a] || !vl[a])) { set_error("fks_op_csr: NULL column or value array"); return FKS_ERR_ARG; }
    for (int64_t q = 0; q < nz; ++q) {
      if (cl[a][q] < 0 || cl[a][q] >= n) { set_error("fks_op_csr: column index out of range"); return FKS_ERR_ARG; }
      if (!std::isfinite(vl[a][q])) { set_error("fks_op_csr: value is NaN/Inf"); return FKS_ERR_ARG; }
    }
  }
  // union pattern, sorted by column within a row, duplicates summed
  std::vector<int64_t> rowptr(n + 1, 0);
  std::vector<int32_t> col;
  std::vector<double> kv, mv;
  std::vector<double> dk(n, 0.0), dm(n, 0.0);
  col.reserve(k_rowptr[n] + m_rowptr[n]);
  kv.reserve(col.capacity());
  mv.reserve(col.capacity());
  std::vector<std::pair<int32_t, int>> ent;  // (column, index into vals)
  std::vector<double> vals;
  for (int64_t i = 0; i < n; ++i) {
    ent.clear();
    vals.clear();
    for (int a = 0; a < 2; ++a)
      for (int64_t q = rp[a][i]; q < rp[a][i + 1]; ++q) {
        ent.push_back({cl[a][q], (int)vals.size() * 2 + a});
        vals.push_back(vl[a][q]);
      }
    std::sort(ent.begin(), ent.end());
    for (size_t e = 0; e < ent.size();) {
      int32_t c = ent[e].first;
      double ks = 0.0, ms = 0.0;
      for (; e < ent.size() && ent[e].first == c; ++e) {
        double v = vals[ent[e].second >> 1];
        if (ent[e].second & 1) ms += v; else ks += v;
      }
      col.push_back(c);
      kv.push_back(ks);
      mv.push_back(ms);
      if (c == i) { dk[i] = ks; dm[i] = ms; }
    }
    rowptr[i + 1] = (int64_t)col.size();
  }
  int64_t nnz = (int64_t)col.size();
  fks_op* op = new fks_op;
  op->ctx = ctx;
  op->dim = 0;
  op->nx = op->ny = op->nz = 0;
  op->n = n;
  op->mask = 0;
  op->csr = true;
  CsrDev& C = op->cd;
  C.nnz = nnz;
  try {
    CK(cudaSetDevice(ctx->device));
    // sliced ELL: each slice of CSR_SLICE rows padded to its longest row
    const int64_t nsl = (n + CSR_SLICE - 1) / CSR_SLICE;
    std::vector<int64_t> sell(nsl + 1, 0);
    std::vector<int32_t> len(n);
    for (int64_t sl = 0; sl < nsl; ++sl) {
      int64_t w = 0;
      for (int64_t r = sl * CSR_SLICE; r < std::min(n, (sl + 1) * CSR_SLICE); ++r) {
        len[r] = (int32_t)(rowptr[r + 1] - rowptr[r]);
        w = std::max<int64_t>(w, len[r]);
      }
      sell[sl + 1] = sell[sl] + w * CSR_SLICE;
    }
    const size_t se = (size_t)std::max<int64_t>(sell[nsl], 1);
    std::vector<int32_t> scol(se, 0);
    std::vector<double> skv(se, 0.0), smv(se, 0.0);
    for (int64_t r = 0; r < n; ++r)
      for (int64_t q = 0; q < len[r]; ++q) {
        const int64_t e = sell[r / CSR_SLICE] + q * CSR_SLICE + (r % CSR_SLICE), src = rowptr[r] + q;
        scol[e] = col[src];
        skv[e] = kv[src];
        smv[e] = mv[src];
      }
    std::vector<float> kf(skv.begin(), skv.end()), mf(smv.begin(), smv.end());
    CK(cudaMalloc(&C.sell, sizeof(int64_t) * (nsl + 1)));
    CK(cudaMalloc(&C.len, sizeof(int32_t) * n));
    CK(cudaMalloc(&C.col, sizeof(int32_t) * se));
    CK(cudaMalloc(&C.kv, sizeof(double) * se));
    CK(cudaMalloc(&C.mv, sizeof(double) * se));
    CK(cudaMalloc(&C.kv32, sizeof(float) * se));
    CK(cudaMalloc(&C.mv32, sizeof(float) * se));
    CK(cudaMalloc(&C.dk, sizeof(double) * n));
    CK(cudaMalloc(&C.dm, sizeof(double) * n));
    CK(cudaMemcpy(C.sell, sell.data(), sizeof(int64_t) * (nsl + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(C.len, len.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(C.col, scol.data(), sizeof(int32_t) * se, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(C.kv, skv.data(), sizeof(double) * se, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(C.mv, smv.data(), sizeof(double) * se, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(C.kv32, kf.data(), sizeof(float) * se, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(C.mv32, mf.data(), sizeof(float) * se, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(C.dk, dk.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(C.dm, dm.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
  } catch (CudaError& e) {
    set_error(std::string("fks_op_csr: ") + e.where + ": " + cudaGetErrorString(e.e));
    fks_op_destroy(op);
    return e.e == cudaErrorMemoryAllocation ? FKS_ERR_OOM : FKS_ERR_CUDA;
  }
  C.dk_h = std::move(dk);
  C.dm_h = std::move(dm);
  C.rowptr_h = std::move(rowptr);
  C.col_h = std::move(col);
  C.kv_h = std::move(kv);
  C.mv_h = std::move(mv);
  *out = op;
  return FKS_OK;
}

void fks_op_destroy(fks_op* op) {
  if (!op) return;
  {
    CsrDev& C = op->cd;
    void* ps[9] = {C.sell, C.len, C.col, C.kv, C.mv, C.kv32, C.mv32, C.dk, C.dm};
    for (void* q : ps)
      if (q) cudaFree(q);
  }
  for (auto& L : op->levels) {
    for (int a = 0; a < 4; ++a) {
      if (L.d64[a]) cudaFree(L.d64[a]);
      if (L.d32[a]) cudaFree(L.d32[a]);
      if (L.d16[a]) cudaFree(L.d16[a]);
      if (L.d32b[a]) cudaFree(L.d32b[a]);
    }
    if (L.kd64) cudaFree(L.kd64);
  }
  if (op->cond_d) cudaFree(op->cond_d);
  op->amg.clear();
  op->lane0.release();
  delete op;
}

int64_t fks_op_size(const fks_op* op) { return op ? op->n : 0; }

fks_status fks_solve(fks_op* op, const fks_c128* b, int n_rhs, const fks_c128* sigma, int n_f, const fks_c128* tau,
                     int n_tau, const fks_options* o, fks_c128* X, double* res_est, double* res_bound,
                     double* res_true, int32_t* m_j, int32_t* shift_status, fks_info* info, void* stream) {
  if (!op || !b || !sigma || !tau || !o || !X || !res_est || !res_bound || !m_j || !shift_status) {
    set_error("fks_solve: NULL argument");
    return FKS_ERR_ARG;
  }
  if (n_rhs < 1 || n_f < 1 || n_tau < 1 || n_tau > MAX_TAU) { set_error("fks_solve: bad n_rhs / n_f / n_tau"); return FKS_ERR_ARG; }
  if ((int64_t)n_f * n_rhs > 65535) { set_error("fks_solve: n_f * n_rhs must be at most 65535"); return FKS_ERR_ARG; }
  if (o->m_max < 1 || o->m_max > MAX_M) { set_error("fks_solve: m_max must be in 1..128"); return FKS_ERR_ARG; }
  if (!(o->tol > 0) || !std::isfinite(o->tol)) { set_error("fks_solve: tol must be positive"); return FKS_ERR_ARG; }
  if (o->variant != FKS_FGMRES && o->variant != FKS_FFOM) { set_error("fks_solve: bad variant"); return FKS_ERR_ARG; }
  if (!prec_ok(o->precision)) { set_error("fks_solve: bad precision"); return FKS_ERR_ARG; }
  if (op->csr && o->precision == FKS_PREC_MIXED_BF16) { set_error("fks_solve: the bf16 smoother option is for grid operators"); return FKS_ERR_ARG; }
  if (o->sched_len < 1 || !o->tau_schedule) { set_error("fks_solve: empty tau schedule"); return FKS_ERR_ARG; }
  for (int i = 0; i < o->sched_len; ++i)
    if (o->tau_schedule[i] < 0 || o->tau_schedule[i] >= n_tau) { set_error("fks_solve: schedule index out of range"); return FKS_ERR_ARG; }
  if (o->launch_mode != 0 && o->launch_mode != 1) { set_error("fks_solve: launch_mode must be 0 or 1"); return FKS_ERR_ARG; }
  if (o->inner_steps > 64) { set_error("fks_solve: inner_steps must be at most 64"); return FKS_ERR_ARG; }
  if (o->assembly != 0 && o->assembly != 1) { set_error("fks_solve: assembly must be 0 or 1"); return FKS_ERR_ARG; }
  if (!std::isfinite(o->inner_relax)) { set_error("fks_solve: inner_relax is not finite"); return FKS_ERR_ARG; }
  if (o->replay_mode && (!o->replay_inner_cycles || !o->replay_mj)) { set_error("fks_solve: replay arrays missing"); return FKS_ERR_ARG; }
  if (o->restart_len < 0 || o->restart_len > o->m_max) { set_error("fks_solve: restart_len must be in 0..m_max"); return FKS_ERR_ARG; }
  if (o->restart_len > 0 && (o->variant != FKS_FFOM || o->replay_mode)) {
    set_error("fks_solve: restarts need the FFOM variant (collinear residuals) and no replay");
    return FKS_ERR_ARG;
  }
  if (o->replay_mode) {
    for (int i = 0; i < o->m_max * n_rhs; ++i)
      if (o->replay_inner_cycles[i] < 0 || o->replay_inner_cycles[i] > 1000) {
        set_error("fks_solve: replay cycle counts must be in 0..1000");
        return FKS_ERR_ARG;
      }
    for (int i = 0; i < n_f * n_rhs; ++i)
      if (o->replay_mj[i] < 1 || o->replay_mj[i] > o->m_max) { set_error("fks_solve: replay m_j out of range"); return FKS_ERR_ARG; }
  }
  // small host-side checks of shifts (device pointers are checked after a copy)
  std::vector<fks_c128> sg(n_f), tu(n_tau);
  cudaMemcpy(sg.data(), sigma, sizeof(fks_c128) * n_f, cudaMemcpyDefault);
  cudaMemcpy(tu.data(), tau, sizeof(fks_c128) * n_tau, cudaMemcpyDefault);
  if (cudaGetLastError() != cudaSuccess) { set_error("fks_solve: cannot read sigma / tau"); return FKS_ERR_ARG; }
  for (auto& z : sg) if (!finite_c(z)) { set_error("fks_solve: sigma has NaN/Inf"); return FKS_ERR_ARG; }
  for (auto& z : tu) if (!finite_c(z)) { set_error("fks_solve: tau has NaN/Inf"); return FKS_ERR_ARG; }
  if (!csr_diag_ok(op, tu.data(), n_tau)) { set_error("fks_solve: K + tau M has a zero diagonal entry"); return FKS_ERR_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  try {
    CK(cudaSetDevice(op->ctx->device));
    if (o->restart_len > 0) {
      if (o->precision == FKS_PREC_FP64)
        return solve_restarted<double>(op, &op->lane0, b, n_rhs, sigma, n_f, tau, n_tau, o, X, res_est, res_bound,
                                       res_true, m_j, shift_status, info, s);
      return solve_restarted<float>(op, &op->lane0, b, n_rhs, sigma, n_f, tau, n_tau, o, X, res_est, res_bound,
                                    res_true, m_j, shift_status, info, s);
    }
    if (o->precision == FKS_PREC_FP64)
      return solve_chunked<double>(op, &op->lane0, b, n_rhs, sigma, n_f, tau, n_tau, o, X, res_est, res_bound, res_true, m_j,
                                   shift_status, info, s);
    return solve_chunked<float>(op, &op->lane0, b, n_rhs, sigma, n_f, tau, n_tau, o, X, res_est, res_bound, res_true, m_j,
                                shift_status, info, s);
  } catch (CudaError& e) {
    set_error(std::string("fks_solve: ") + e.where + ": " + cudaGetErrorString(e.e));
    return e.e == cudaErrorMemoryAllocation ? FKS_ERR_OOM : FKS_ERR_CUDA;
  }
}

fks_status fks_op_set_fusion(fks_op* op, int precision, int64_t max_cells) {
  if (!op) { set_error("fks_op_set_fusion: NULL operator"); return FKS_ERR_ARG; }
  if (op->csr) { set_error("fks_op_set_fusion: grid operators only"); return FKS_ERR_ARG; }
  if (!prec_ok(precision)) { set_error("fks_op_set_fusion: bad precision"); return FKS_ERR_ARG; }
  op->fuse_max[precision == FKS_PREC_FP64 ? 0 : 1] = max_cells < 0 ? INT64_MAX : max_cells;
  return FKS_OK;
}

fks_status fks_op_set_tiles(fks_op* op, int precision, int64_t max_cells) {
  if (!op) { set_error("fks_op_set_tiles: NULL operator"); return FKS_ERR_ARG; }
  if (op->csr) { set_error("fks_op_set_tiles: grid operators only"); return FKS_ERR_ARG; }
  if (!prec_ok(precision)) { set_error("fks_op_set_tiles: bad precision"); return FKS_ERR_ARG; }
  op->tile16_max[precision == FKS_PREC_FP64 ? 0 : 1] = max_cells < 0 ? INT64_MAX : max_cells;
  return FKS_OK;
}

fks_status fks_op_set_tiles8(fks_op* op, int precision, int64_t max_cells) {
  if (!op) { set_error("fks_op_set_tiles8: NULL operator"); return FKS_ERR_ARG; }
  if (op->csr) { set_error("fks_op_set_tiles8: grid operators only"); return FKS_ERR_ARG; }
  if (!prec_ok(precision)) { set_error("fks_op_set_tiles8: bad precision"); return FKS_ERR_ARG; }
  op->tile8_max[precision == FKS_PREC_FP64 ? 0 : 1] = max_cells < 0 ? INT64_MAX : max_cells;
  return FKS_OK;
}

fks_status fks_op_set_tail(fks_op* op, int precision, int64_t max_cells) {
  if (!op) { set_error("fks_op_set_tail: NULL operator"); return FKS_ERR_ARG; }
  if (op->csr) { set_error("fks_op_set_tail: grid operators only"); return FKS_ERR_ARG; }
  if (!prec_ok(precision)) { set_error("fks_op_set_tail: bad precision"); return FKS_ERR_ARG; }
  if (max_cells < 1) { set_error("fks_op_set_tail: max_cells must be >= 1"); return FKS_ERR_ARG; }
  int lt;
  size_t smem;
  if (precision == FKS_PREC_FP64) {
    lt = tail_level<double>(op->levels, max_cells);
    smem = tail_smem<double>(op->levels, lt);
  } else {
    lt = tail_level<float>(op->levels, max_cells);
    smem = tail_smem<float>(op->levels, lt);
  }
  if (smem > TAIL_SMEM_LIMIT) { set_error("fks_op_set_tail: the tail levels do not fit in shared memory"); return FKS_ERR_ARG; }
  op->tail_max[precision == FKS_PREC_FP64 ? 0 : 1] = max_cells;
  return FKS_OK;
}

fks_status fks_op_set_cluster(fks_op* op, int precision, int64_t max_cells) {
  if (!op) { set_error("fks_op_set_cluster: NULL operator"); return FKS_ERR_ARG; }
  if (op->csr) { set_error("fks_op_set_cluster: grid operators only"); return FKS_ERR_ARG; }
  if (!prec_ok(precision)) { set_error("fks_op_set_cluster: bad precision"); return FKS_ERR_ARG; }
  const int pi = precision == FKS_PREC_FP64 ? 0 : 1;
  if (max_cells <= 0) {
    op->cluster_max[pi] = 0;
    return FKS_OK;
  }
  size_t smem = 0;
  bool ok;
  try {
    CK(cudaSetDevice(op->ctx->device));
    if (precision == FKS_PREC_FP64) {
      ok = cluster_level_for<double>(op->levels, max_cells, nullptr, &smem) >= 0;
      if (ok) {
        std::lock_guard<std::mutex> build_lock(g_build_mu);
        ok = cluster_launchable<double>(smem);
      }
    } else {
      ok = cluster_level_for<float>(op->levels, max_cells, nullptr, &smem) >= 0;
      if (ok) {
        std::lock_guard<std::mutex> build_lock(g_build_mu);
        ok = cluster_launchable<float>(smem);
      }
    }
  } catch (CudaError& e) {
    set_error(std::string("fks_op_set_cluster: ") + e.where + ": " + cudaGetErrorString(e.e));
    return FKS_ERR_CUDA;
  }
  if (!ok) {
    set_error("fks_op_set_cluster: no level qualifies for the cluster V-cycle, or its cluster cannot be scheduled");
    return FKS_ERR_ARG;
  }
  op->cluster_max[pi] = max_cells;
  return FKS_OK;
}

fks_status fks_op_set_coop(fks_op* op, int precision, int64_t max_cells) {
  if (!op) { set_error("fks_op_set_coop: NULL operator"); return FKS_ERR_ARG; }
  if (!prec_ok(precision)) { set_error("fks_op_set_coop: bad precision"); return FKS_ERR_ARG; }
  if (max_cells < 0) { set_error("fks_op_set_coop: max_cells must be >= 0"); return FKS_ERR_ARG; }
  op->coop_max[precision == FKS_PREC_FP64 ? 0 : 1] = max_cells;
  return FKS_OK;
}

fks_status fks_op_coop_max(fks_op* op, int precision, int64_t* max_cells) {
  if (!op || !max_cells) { set_error("fks_op_coop_max: NULL argument"); return FKS_ERR_ARG; }
  if (!prec_ok(precision)) { set_error("fks_op_coop_max: bad precision"); return FKS_ERR_ARG; }
  *max_cells = op->coop_max[precision == FKS_PREC_FP64 ? 0 : 1];
  return FKS_OK;
}

int fks_set_pdl(int on) {
  const int prev = fks::pdl_flag();
  if (on >= 0) fks::pdl_flag() = on ? 1 : 0;
  return prev;
}

fks_status fks_op_set_zchunk(fks_op* op, int precision, int level, int planes) {
  if (!op) { set_error("fks_op_set_zchunk: NULL operator"); return FKS_ERR_ARG; }
  if (op->csr) { set_error("fks_op_set_zchunk: grid operators only"); return FKS_ERR_ARG; }
  if (!prec_ok(precision)) { set_error("fks_op_set_zchunk: bad precision"); return FKS_ERR_ARG; }
  if (level < 0 || level >= (int)op->levels.size()) { set_error("fks_op_set_zchunk: no such level"); return FKS_ERR_ARG; }
  op->zchunk[precision == FKS_PREC_FP64 ? 0 : 1][level] = planes <= 0 ? 0 : std::max(2, planes & ~1);
  return FKS_OK;
}

fks_status fks_op_zchunks(const fks_op* op, int precision, int32_t* planes, int cap, int* levels) {
  if (!op) { set_error("fks_op_zchunks: NULL operator"); return FKS_ERR_ARG; }
  if (!prec_ok(precision)) { set_error("fks_op_zchunks: bad precision"); return FKS_ERR_ARG; }
  const int nl = (int)op->levels.size();
  if (levels) *levels = nl;
  for (int l = 0; l < nl && l < cap && planes; ++l) planes[l] = op->zchunk[precision == FKS_PREC_FP64 ? 0 : 1][l];
  return FKS_OK;
}

fks_status fks_op_tiling(const fks_op* op, int precision, int64_t* fuse_max, int64_t* tile16_max,
                         int64_t* tail_max, int64_t* cluster_max, int64_t* tile8_max) {
  if (!op) { set_error("fks_op_tiling: NULL operator"); return FKS_ERR_ARG; }
  if (!prec_ok(precision)) { set_error("fks_op_tiling: bad precision"); return FKS_ERR_ARG; }
  int pi = precision == FKS_PREC_FP64 ? 0 : 1;
  if (fuse_max) *fuse_max = op->fuse_max[pi];
  if (tile16_max) *tile16_max = op->tile16_max[pi];
  if (tail_max) *tail_max = op->tail_max[pi];
  if (cluster_max) *cluster_max = op->cluster_max[pi];
  if (tile8_max) *tile8_max = op->tile8_max[pi];
  return FKS_OK;
}

fks_status fks_op_autotune(fks_op* op, int precision, fks_c128 tau, void* stream, int64_t* chosen) {
  if (!op) { set_error("fks_op_autotune: NULL operator"); return FKS_ERR_ARG; }
  if (op->csr) { set_error("fks_op_autotune: grid operators only"); return FKS_ERR_ARG; }
  if (!prec_ok(precision)) { set_error("fks_op_autotune: bad precision"); return FKS_ERR_ARG; }
  if (!finite_c(tau)) { set_error("fks_op_autotune: tau has NaN/Inf"); return FKS_ERR_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  int pi = precision == FKS_PREC_FP64 ? 0 : 1;
  int64_t saved = op->fuse_max[pi], saved16 = op->tile16_max[pi], savedt = op->tail_max[pi];
  int64_t savedc = op->cluster_max[pi], saved8 = op->tile8_max[pi], savedco = op->coop_max[pi];
  int savedz[MAX_LEVELS];
  std::memcpy(savedz, op->zchunk[pi], sizeof(savedz));
  try {
    CK(cudaSetDevice(op->ctx->device));
    Solve S{};
    S.op = op;
    S.lane = &op->lane0;
    S.s = s;
    S.nslot = 1;
    S.n_f = 1;
    S.n_tau = 1;
    S.m = 1;
    S.sched_len = 1;
    S.precision = precision;
    S.n = op->n;
    S.eps = 1e-30;
    S.max_cycles = 1;
    SlotState sh{};
    S.st_host = &sh;
    auto run = [&](auto tag) {
      using VT = decltype(tag);
      Arena probe;
      carve<VT>(S, probe, false);
      op->lane0.ws.reserve(probe.off + 4096);
      carve<VT>(S, op->lane0.ws, false);
      const LevelHost& L0 = op->levels[0];
      CK(cudaMemcpyAsync(S.taus, &tau, sizeof(z64), cudaMemcpyHostToDevice, s));
      SlotState st0{};
      st0.active = 1;
      st0.k = 1;
      CK(cudaMemcpyAsync(S.st, &st0, sizeof(SlotState), cudaMemcpyHostToDevice, s));
      CK(cudaMemsetAsync(S.f[0], 0, sizeof(cx<VT>) * L0.n, s));
      setup_levels<VT>(S);
      // candidate thresholds that change which levels are fused
      std::vector<int64_t> cand = {0};
      for (auto& L : op->levels)
        if (fused_level_ok(L) || fused3d_level_ok(L)) cand.push_back(L.n);
      std::sort(cand.begin(), cand.end());
      cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
      cudaStream_t cs = nullptr;
      CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaEvent_t e0, e1;
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
      double best = 1e30;
      int64_t pick = saved, pick16 = saved16, pickt = savedt, pickc = savedc, pick8 = 0;
      op->coop_max[pi] = 0;  // the other choices are timed without the cooperative lower cycle
      struct Choice { int64_t fuse, t16, tail, cl, t8; };
      std::vector<Choice> choices;
      // fusion choices for the levels above the single-launch lower part
      // starting at level ls (thresholds below those levels' sizes are all "none")
      auto add = [&](int ls, int64_t tm, int64_t cm) {
        std::vector<int64_t> cs = {0};
        for (int64_t c : cand)
          if (c > op->levels[ls].n) cs.push_back(c);
        for (int64_t c : cs)
          for (int64_t t : cs)
            if (t <= c) choices.push_back({c, t, tm, cm, 0});
      };
      for (int64_t tm : {int64_t(64), int64_t(256), int64_t(1024), int64_t(4096)}) {
        const int lt = tail_level<VT>(op->levels, tm);
        if (tail_smem<VT>(op->levels, lt) > TAIL_SMEM_LIMIT) continue;  // f and z must fit
        add(lt, tm, 0);
      }
      // the cluster kernel from every level where it applies, down to 1024 cells
      for (size_t l = 0; l + 1 < op->levels.size(); ++l) {
        const int64_t cm = op->levels[l].n;
        if (cm < 1024) break;
        size_t csm = 0;
        if (cluster_level_for<VT>(op->levels, cm, nullptr, &csm) != (int)l) continue;
        bool ok;
        {
          std::lock_guard<std::mutex> build_lock(g_build_mu);
          ok = cluster_launchable<VT>(csm);
        }
        if (ok) add((int)l, savedt, cm);
      }
      auto measure = [&](const Choice& ch) -> float {
        op->fuse_max[pi] = ch.fuse;
        op->tile16_max[pi] = ch.t16;
        op->tail_max[pi] = ch.tail;
        op->cluster_max[pi] = ch.cl;
        op->tile8_max[pi] = ch.t8;
        {
          // the tail's shared memory and coefficient blob follow the threshold
          std::lock_guard<std::mutex> build_lock(g_build_mu);
          tail_prepare<VT>(tail_launch_smem<VT>(op->levels, tail_level<VT>(op->levels, ch.tail)));
        }
        Arena probe2;
        carve<VT>(S, probe2, false);
        op->lane0.ws.reserve(probe2.off + 4096);
        carve<VT>(S, op->lane0.ws, false);
        CK(cudaMemcpyAsync(S.taus, &tau, sizeof(z64), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(S.st, &st0, sizeof(SlotState), cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(S.f[0], 0, sizeof(cx<VT>) * L0.n, s));
        setup_levels<VT>(S);
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        S.s = cs;
        S.capturing = true;
        int64_t keep = op->lane0.prof.all_launches;
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        vcycle<VT>(S);
        CK(cudaStreamEndCapture(cs, &g));
        op->lane0.prof.all_launches = keep;
        S.capturing = false;
        S.s = s;
        CK(cudaGraphInstantiate(&ge, g, 0));
        for (int w = 0; w < 3; ++w) CK(cudaGraphLaunch(ge, s));
        const int reps = 10;
        CK(cudaEventRecord(e0, s));
        for (int w = 0; w < reps; ++w) CK(cudaGraphLaunch(ge, s));
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        cudaGraphExecDestroy(ge);
        cudaGraphDestroy(g);
        return ms;
      };
      for (const Choice& ch : choices) {
        const float ms = measure(ch);
        if (ms < best) {
          best = ms;
          pick = ch.fuse;
          pick16 = ch.t16;
          pickt = ch.tail;
          pickc = ch.cl;
        }
      }
      // then 8 x 8 tiles for the smallest fused levels of the pick
      for (int64_t u : cand) {
        if (u == 0 || u > pick16 || u > pick) continue;
        const float ms = measure({pick, pick16, pickt, pickc, u});
        if (ms < best) {
          best = ms;
          pick8 = u;
        }
      }
      // then the z-chunk of every fused 3D level of the pick, level by level
      {
        const Choice ch{pick, pick16, pickt, pickc, pick8};
        const int lt = tail_level<VT>(op->levels, pickt);
        for (int l = 0; l < lt && l < MAX_LEVELS; ++l) {
          const LevelHost& L = op->levels[l];
          if (!fused3d_level_ok(L) || L.n > pick) continue;
          int bestz = op->zchunk[pi][l];
          for (int zc : {2, 4, 8, 16, 32, 64, 0}) {
            if (zc > L.nz || zc == bestz) continue;
            op->zchunk[pi][l] = zc;
            const float ms = measure(ch);
            if (ms < best) {
              best = ms;
              bestz = zc;
            }
          }
          op->zchunk[pi][l] = bestz;
        }
      }
      // then the cooperative lower cycle from each level above the pick's tail
      {
        const Choice ch{pick, pick16, pickt, pickc, pick8};
        int64_t pickco = 0;
        if (pickc == 0 && coop_capacity_vcycle<VT>() > 0) {
          const int lt = tail_level<VT>(op->levels, pickt);
          for (int l = 1; l < lt; ++l) {
            op->coop_max[pi] = op->levels[l].n;
            const float ms = measure(ch);
            if (ms < best) {
              best = ms;
              pickco = op->levels[l].n;
            }
          }
        }
        op->coop_max[pi] = pickco;
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      cudaStreamDestroy(cs);
      op->fuse_max[pi] = pick;
      op->tile16_max[pi] = pick16;
      op->tail_max[pi] = pickt;
      op->cluster_max[pi] = pickc;
      op->tile8_max[pi] = pick8;
    };
    if (precision == FKS_PREC_FP64) run(double{});
    else run(float{});
  } catch (CudaError& e) {
    op->fuse_max[pi] = saved;
    op->tile16_max[pi] = saved16;
    op->tail_max[pi] = savedt;
    op->cluster_max[pi] = savedc;
    op->tile8_max[pi] = saved8;
    op->coop_max[pi] = savedco;
    std::memcpy(op->zchunk[pi], savedz, sizeof(savedz));
    set_error(std::string("fks_op_autotune: ") + e.where + ": " + cudaGetErrorString(e.e));
    return FKS_ERR_CUDA;
  }
  if (chosen) *chosen = op->fuse_max[pi];
  return FKS_OK;
}

fks_status fks_profile_select(fks_op* op, int kclass, int level) {
  if (!op) { set_error("fks_profile_select: NULL operator"); return FKS_ERR_ARG; }
  if (kclass >= FKS_K_COUNT) { set_error("fks_profile_select: bad kernel class"); return FKS_ERR_ARG; }
  op->lane0.prof.cls = kclass < 0 ? -1 : kclass;
  op->lane0.prof.level = level;
  return FKS_OK;
}

fks_status fks_profile_read(fks_op* op, int64_t* launches, double* total_ms, double* alg_bytes, double* alg_flops,
                            int64_t* all_launches) {
  if (!op) { set_error("fks_profile_read: NULL operator"); return FKS_ERR_ARG; }
  Prof& p = op->lane0.prof;
  p.collect();
  if (launches) *launches = p.launches;
  if (total_ms) *total_ms = p.ms;
  if (alg_bytes) *alg_bytes = p.tot_bytes;
  if (alg_flops) *alg_flops = p.tot_flops;
  if (all_launches) *all_launches = p.all_launches;
  p.launches = 0;
  p.ms = 0;
  p.tot_bytes = 0;
  p.tot_flops = 0;
  p.all_launches = 0;
  return FKS_OK;
}

fks_status fks_op_apply(fks_op* op, fks_c128 sh, const fks_c128* x, fks_c128* y, int n_vec, void* stream) {
  if (!op || !x || !y || n_vec < 1 || n_vec > 65535) { set_error("fks_op_apply: bad argument"); return FKS_ERR_ARG; }
  if (!finite_c(sh)) { set_error("fks_op_apply: shift has NaN/Inf"); return FKS_ERR_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  try {
    CK(cudaSetDevice(op->ctx->device));
    int64_t n = op->n;
    bool xd = is_device_ptr(x), yd = is_device_ptr(y);
    size_t bytes = sizeof(z64) * n * n_vec;
    Arena& A = op->lane0.ws;
    A.reserve(2 * bytes + 1024);
    A.reset();
    z64* xs = xd ? (z64*)x : A.take<z64>((size_t)n * n_vec);
    z64* ys = yd ? (z64*)y : A.take<z64>((size_t)n * n_vec);
    if (!xd) CK(cudaMemcpyAsync(xs, x, bytes, cudaMemcpyHostToDevice, s));
    if (op->csr)
      launch_csr_apply<double>(op->cd.view<double>(n), mk(sh.re, sh.im), nullptr, nullptr, xs, ys, n, n_vec, s);
    else
      launch_apply<double>(op->levels[0], mk(sh.re, sh.im), nullptr, nullptr, xs, ys, n, n_vec, s);
    CK(cudaGetLastError());
    if (!yd) CK(cudaMemcpyAsync(y, ys, bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  } catch (CudaError& e) {
    set_error(std::string("fks_op_apply: ") + e.where + ": " + cudaGetErrorString(e.e));
    return FKS_ERR_CUDA;
  }
  return FKS_OK;
}

fks_status fks_op_amg(fks_op* op, int enable, int max_levels, int64_t max_coarse, int nu) {
  if (!op || !op->csr) { set_error("fks_op_amg: needs a CSR operator"); return FKS_ERR_ARG; }
  if (max_levels < 0 || max_levels > AMG_MAX_LEVELS || max_coarse < 0 || max_coarse > AMG_MAX_DENSE || nu < 0 ||
      nu > 8) {
    set_error("fks_op_amg: need 0 <= max_levels <= 16, 0 <= max_coarse <= 4096, 0 <= nu <= 8");
    return FKS_ERR_ARG;
  }
  try {
    CK(cudaSetDevice(op->ctx->device));
    std::lock_guard<std::mutex> lock(op->amg.mu);
    op->amg.clear();
    op->amg.on = enable != 0;
    op->amg.max_levels = max_levels ? max_levels : 10;
    op->amg.max_coarse = max_coarse ? max_coarse : 256;
    op->amg.nu = nu ? nu : 2;
    op->amg.gen++;
  } catch (CudaError& e) {
    set_error(std::string("fks_op_amg: ") + e.where + ": " + cudaGetErrorString(e.e));
    return FKS_ERR_CUDA;
  }
  return FKS_OK;
}

fks_status fks_op_amg_setup(fks_op* op, const fks_c128* tau, int n_tau, int precision, double* setup_ms) {
  if (!op || !tau || !op->csr || !op->amg.on) { set_error("fks_op_amg_setup: needs a CSR operator with AMG on"); return FKS_ERR_ARG; }
  if (n_tau < 1 || n_tau > MAX_TAU) { set_error("fks_op_amg_setup: n_tau must be in 1..16"); return FKS_ERR_ARG; }
  if (precision != FKS_PREC_FP64 && precision != FKS_PREC_MIXED) { set_error("fks_op_amg_setup: bad precision (the bf16 option is for grid operators)"); return FKS_ERR_ARG; }
  for (int q = 0; q < n_tau; ++q)
    if (!finite_c(tau[q])) { set_error("fks_op_amg_setup: tau has NaN/Inf"); return FKS_ERR_ARG; }
  if (!csr_diag_ok(op, tau, n_tau)) { set_error("fks_op_amg_setup: K + tau M has a zero diagonal entry"); return FKS_ERR_ARG; }
  try {
    CK(cudaSetDevice(op->ctx->device));
    std::string err;
    if (precision == FKS_PREC_FP64) {
      std::vector<AmgLevel<double>> t;
      err = amg_ensure<double>(op, tau, n_tau, &t, setup_ms);
    } else {
      std::vector<AmgLevel<float>> t;
      err = amg_ensure<float>(op, tau, n_tau, &t, setup_ms);
    }
    if (!err.empty()) { set_error("fks_op_amg_setup: " + err); return FKS_ERR_ARG; }
  } catch (CudaError& e) {
    set_error(std::string("fks_op_amg_setup: ") + e.where + ": " + cudaGetErrorString(e.e));
    return e.e == cudaErrorMemoryAllocation ? FKS_ERR_OOM : FKS_ERR_CUDA;
  }
  return FKS_OK;
}

fks_status fks_op_amg_info(fks_op* op, int* n_levels, int64_t* sizes, int sizes_cap, int32_t* agg, int64_t agg_cap) {
  if (!op || !n_levels || !op->csr) { set_error("fks_op_amg_info: needs a CSR operator"); return FKS_ERR_ARG; }
  std::lock_guard<std::mutex> lock(op->amg.mu);
  const AmgState& M = op->amg;
  if (M.sizes.empty()) { set_error("fks_op_amg_info: no hierarchy built yet"); return FKS_ERR_ARG; }
  const int L = (int)M.sizes.size();
  *n_levels = L;
  if (sizes) {
    if (sizes_cap < L) { set_error("fks_op_amg_info: sizes_cap too small"); return FKS_ERR_ARG; }
    for (int l = 0; l < L; ++l) sizes[l] = M.sizes[l];
  }
  if (agg) {
    int64_t need = 0;
    for (const auto& a : M.agg.agg) need += (int64_t)a.size();
    if (agg_cap < need) { set_error("fks_op_amg_info: agg_cap too small"); return FKS_ERR_ARG; }
    int64_t at = 0;
    for (const auto& a : M.agg.agg) {
      std::memcpy(agg + at, a.data(), sizeof(int32_t) * a.size());
      at += (int64_t)a.size();
    }
  }
  return FKS_OK;
}

fks_status fks_amg_host_shape(int64_t n, const int64_t* rowptr, const int32_t* col, const fks_c128* val,
                              int max_levels, int64_t max_coarse, int* n_levels, int64_t* sizes, int64_t* nnz_a,
                              int64_t* nnz_p, double* omega, int sizes_cap, int32_t* agg, int64_t agg_cap) {
  if (!rowptr || !n_levels || n < 1 || n > INT32_MAX) { set_error("fks_amg_host_shape: bad arguments"); return FKS_ERR_ARG; }
  if (max_levels < 0 || max_levels > AMG_MAX_LEVELS || max_coarse < 0 || max_coarse > AMG_MAX_DENSE) {
    set_error("fks_amg_host_shape: need 0 <= max_levels <= 16, 0 <= max_coarse <= 4096");
    return FKS_ERR_ARG;
  }
  if (rowptr[0] != 0) { set_error("fks_amg_host_shape: row pointers must start at 0"); return FKS_ERR_ARG; }
  AmgCsr A;
  A.n = A.m = n;
  A.rp.assign(rowptr, rowptr + n + 1);
  for (int64_t i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) { set_error("fks_amg_host_shape: row pointers must not decrease"); return FKS_ERR_ARG; }
    for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
      if (col[q] < 0 || col[q] >= n || (q > rowptr[i] && col[q] <= col[q - 1])) {
        set_error("fks_amg_host_shape: columns must be in range and ascending within a row");
        return FKS_ERR_ARG;
      }
      if (!finite_c(val[q])) { set_error("fks_amg_host_shape: value is NaN/Inf"); return FKS_ERR_ARG; }
    }
  }
  const int64_t nnz = rowptr[n];
  A.ci.assign(col, col + nnz);
  A.v.resize(nnz);
  for (int64_t q = 0; q < nnz; ++q) A.v[q] = mk(val[q].re, val[q].im);
  AmgAgg ag;
  AmgHost h;
  std::string err = amg_build(A, max_levels ? max_levels : 10, max_coarse ? max_coarse : 256, &ag, &h);
  if (!err.empty()) { set_error("fks_amg_host_shape: " + err); return FKS_ERR_ARG; }
  const int L = (int)h.lv.size();
  *n_levels = L;
  if (sizes_cap < L && (sizes || nnz_a || nnz_p || omega)) { set_error("fks_amg_host_shape: sizes_cap too small"); return FKS_ERR_ARG; }
  for (int l = 0; l < L; ++l) {
    if (sizes) sizes[l] = h.lv[l].A.n;
    if (nnz_a) nnz_a[l] = (int64_t)h.lv[l].A.ci.size();
    if (nnz_p) nnz_p[l] = (int64_t)h.lv[l].P.ci.size();
    if (omega) omega[l] = h.lv[l].omega;
  }
  if (agg) {
    int64_t need = 0;
    for (const auto& a : ag.agg) need += (int64_t)a.size();
    if (agg_cap < need) { set_error("fks_amg_host_shape: agg_cap too small"); return FKS_ERR_ARG; }
    int64_t at = 0;
    for (const auto& a : ag.agg) {
      std::memcpy(agg + at, a.data(), sizeof(int32_t) * a.size());
      at += (int64_t)a.size();
    }
  }
  return FKS_OK;
}

fks_status fks_ritz(fks_ctx* ctx, const fks_c128* hbar, const fks_c128* tau_k, const int32_t* steps, int n_rhs,
                    int m_max, fks_c128* theta, int32_t* status, void* stream) {
  if (!ctx || !hbar || !tau_k || !steps || !theta || !status) { set_error("fks_ritz: NULL argument"); return FKS_ERR_ARG; }
  if (n_rhs < 1 || m_max < 1 || m_max > MAX_M) { set_error("fks_ritz: need n_rhs >= 1 and 1 <= m_max <= 128"); return FKS_ERR_ARG; }
  if (!is_device_ptr(steps))
    for (int r = 0; r < n_rhs; ++r)
      if (steps[r] < 0 || steps[r] > m_max) { set_error("fks_ritz: steps outside [0, m_max]"); return FKS_ERR_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nh = (size_t)(m_max + 1) * m_max * n_rhs, nt = (size_t)m_max * n_rhs;
  std::vector<void*> owned;
  auto dev = [&](const void* p, size_t bytes) -> void* {
    if (is_device_ptr(p)) return (void*)p;
    void* d = nullptr;
    CK(cudaMallocAsync(&d, bytes, s));
    owned.push_back(d);
    CK(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, s));
    return d;
  };
  fks_status ret = FKS_OK;
  try {
    CK(cudaSetDevice(ctx->device));
    const z64* hd = (const z64*)dev(hbar, sizeof(z64) * nh);
    const z64* td = (const z64*)dev(tau_k, sizeof(z64) * nt);
    const int32_t* sd = (const int32_t*)dev(steps, sizeof(int32_t) * n_rhs);
    z64* scratch = nullptr;
    CK(cudaMallocAsync((void**)&scratch, sizeof(z64) * 2 * (size_t)n_rhs * m_max * m_max, s));
    owned.push_back(scratch);
    z64* thd = is_device_ptr(theta) ? (z64*)theta : nullptr;
    if (!thd) { CK(cudaMallocAsync((void**)&thd, sizeof(z64) * nt, s)); owned.push_back(thd); }
    int32_t* std_ = is_device_ptr(status) ? status : nullptr;
    if (!std_) { CK(cudaMallocAsync((void**)&std_, sizeof(int32_t) * n_rhs, s)); owned.push_back(std_); }
    launch_ritz(hd, td, sd, n_rhs, m_max, scratch, thd, std_, s);
    CK(cudaGetLastError());
    if (thd != (z64*)theta) CK(cudaMemcpyAsync(theta, thd, sizeof(z64) * nt, cudaMemcpyDeviceToHost, s));
    if (std_ != status) CK(cudaMemcpyAsync(status, std_, sizeof(int32_t) * n_rhs, cudaMemcpyDeviceToHost, s));
    for (void* p : owned) cudaFreeAsync(p, s);
    owned.clear();
    CK(cudaStreamSynchronize(s));
  } catch (CudaError& e) {
    for (void* p : owned) cudaFreeAsync(p, s);
    set_error(std::string("fks_ritz: ") + e.where + ": " + cudaGetErrorString(e.e));
    ret = e.e == cudaErrorMemoryAllocation ? FKS_ERR_OOM : FKS_ERR_CUDA;
  }
  return ret;
}

fks_status fks_sensitivity(fks_op* op, const fks_c128* phi, const fks_c128* psi, int n_m, const fks_c128* sigma,
                           int n_f, fks_c128* j_lnk, fks_c128* j_lns, void* stream) {
  if (!op || !phi || !psi || !sigma || !j_lnk || !j_lns) { set_error("fks_sensitivity: NULL argument"); return FKS_ERR_ARG; }
  if (op->csr || !op->cond_d) { set_error("fks_sensitivity: grid operators only"); return FKS_ERR_ARG; }
  if (n_m < 1 || n_f < 1 || n_f > 65535) { set_error("fks_sensitivity: need n_m >= 1 and 1 <= n_f <= 65535"); return FKS_ERR_ARG; }
  if (!is_device_ptr(sigma))
    for (int j = 0; j < n_f; ++j)
      if (!finite_c(sigma[j])) { set_error("fks_sensitivity: sigma has NaN/Inf"); return FKS_ERR_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  try {
    CK(cudaSetDevice(op->ctx->device));
    const int64_t n = op->n;
    const size_t blk = sizeof(z64) * (size_t)n * n_f;  // one measurement's n_f phasors
    const bool all_dev = is_device_ptr(phi) && is_device_ptr(psi) && is_device_ptr(j_lnk) && is_device_ptr(j_lns);
    Arena& A = op->lane0.ws;
    const size_t need = (all_dev ? 0 : 4 * blk) + sizeof(z64) * n_f + 8192;
    A.reserve(need);
    A.reset();
    z64* sg = A.take<z64>(n_f);
    copy_in(sg, sigma, sizeof(z64) * n_f, s);
    if (all_dev) {
      launch_sensitivity(op->levels[0], op->cond_d, (const z64*)phi, (const z64*)psi, n_m, n_f, sg, (z64*)j_lnk,
                         (z64*)j_lns, s);
      CK(cudaGetLastError());
    } else {
      // one measurement at a time through device staging buffers
      z64* ph = A.take<z64>((size_t)n * n_f);
      z64* ps = A.take<z64>((size_t)n * n_f);
      z64* jk = A.take<z64>((size_t)n * n_f);
      z64* js = A.take<z64>((size_t)n * n_f);
      copy_in(ph, phi, blk, s);
      for (int m = 0; m < n_m; ++m) {
        copy_in(ps, psi + (size_t)m * n * n_f, blk, s);
        launch_sensitivity(op->levels[0], op->cond_d, ph, ps, 1, n_f, sg, jk, js, s);
        CK(cudaGetLastError());
        copy_out(j_lnk + (size_t)m * n * n_f, jk, blk, s);
        copy_out(j_lns + (size_t)m * n * n_f, js, blk, s);
      }
    }
    CK(cudaStreamSynchronize(s));
  } catch (CudaError& e) {
    set_error(std::string("fks_sensitivity: ") + e.where + ": " + cudaGetErrorString(e.e));
    return e.e == cudaErrorMemoryAllocation ? FKS_ERR_OOM : FKS_ERR_CUDA;
  }
  return FKS_OK;
}

fks_status fks_precond_apply(fks_op* op, fks_c128 tau, const fks_c128* v, fks_c128* z, double eps, int max_cycles,
                             int cycles, int precision, int32_t* out_cycles, double* out_pnorm, void* stream) {
  if (!op || !v || !z) { set_error("fks_precond_apply: NULL argument"); return FKS_ERR_ARG; }
  if (!finite_c(tau)) { set_error("fks_precond_apply: tau has NaN/Inf"); return FKS_ERR_ARG; }
  if (!prec_ok(precision)) { set_error("fks_precond_apply: bad precision"); return FKS_ERR_ARG; }
  if (cycles < 0 && !(eps > 0)) { set_error("fks_precond_apply: eps must be positive"); return FKS_ERR_ARG; }
  if (!csr_diag_ok(op, &tau, 1)) { set_error("fks_precond_apply: K + tau M has a zero diagonal entry"); return FKS_ERR_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  try {
    CK(cudaSetDevice(op->ctx->device));
    Solve S{};
    S.op = op;
    S.lane = &op->lane0;
    S.s = s;
    S.nslot = 1;
    S.n_f = 1;
    S.n_tau = 1;
    S.m = 1;
    S.sched_len = 1;
    S.precision = precision;
    S.n = op->n;
    S.eps = eps;
    S.max_cycles = max_cycles > 0 ? max_cycles : 50;
    S.replay = cycles >= 0;
    S.inner_steps = op->csr && op->amg.on ? 4 : 8;
    std::string amg_err;
    auto run = [&](auto tag) {
      using VT = decltype(tag);
      amg_err = amg_prepare<VT>(S, &tau);
      if (!amg_err.empty()) return;
      Arena probe;
      carve<VT>(S, probe, false);
      op->lane0.ws.reserve(probe.off + 4096);
      carve<VT>(S, op->lane0.ws, false);
      if (S.amg)
        CK(cudaMemcpyAsync(S.amg_tab, S.amg_table.data(), S.amg_table.size(), cudaMemcpyHostToDevice, s));
      int64_t n = S.n;
      copy_in(S.V, v, sizeof(z64) * n, s);
      // z = 0 when no cycle runs (a replayed count of 0, or v = 0 in the eps mode)
      CK(cudaMemsetAsync(S.Z, 0, sizeof(z64) * n, s));
      CK(cudaMemcpyAsync(S.taus, &tau, sizeof(z64), cudaMemcpyHostToDevice, s));
      int32_t cyc = cycles;
      CK(cudaMemcpyAsync(S.rep_cyc, &cyc, sizeof(int32_t), cudaMemcpyHostToDevice, s));
      SlotState st0{};
      st0.active = 1;
      st0.k = 1;
      st0.tau = 0;
      CK(cudaMemcpyAsync(S.st, &st0, sizeof(SlotState), cudaMemcpyHostToDevice, s));
      std::vector<SlotState> sh(1);
      S.st_host = sh.data();
      setup_levels<VT>(S);
      inner_solve<VT>(S, S.V, n, S.Z, n);
      CK(cudaGetLastError());
      copy_out(z, S.Z, sizeof(z64) * n, s);
      CK(cudaMemcpyAsync(S.st_host, S.st, sizeof(SlotState), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (out_cycles) *out_cycles = S.st_host[0].cycles;
      if (out_pnorm) *out_pnorm = std::sqrt(S.st_host[0].pnorm2);
    };
    if (precision == FKS_PREC_FP64) run(double{});
    else run(float{});
    if (!amg_err.empty()) {
      set_error("fks_precond_apply: " + amg_err);
      return FKS_ERR_ARG;
    }
  } catch (CudaError& e) {
    set_error(std::string("fks_precond_apply: ") + e.where + ": " + cudaGetErrorString(e.e));
    return e.e == cudaErrorMemoryAllocation ? FKS_ERR_OOM : FKS_ERR_CUDA;
  }
  return FKS_OK;
}

}  // extern "C"

// ====================================================================== allocation-free preconditioner apply
// For callers that may not allocate device memory: code running inside a host
// framework whose memory pool owns all of the GPU's memory, or code that cannot
// afford cudaMalloc's implicit device synchronisation in a real-time loop. The
// multigrid scratch lives in one fixed file-scope device array instead of the
// operator's workspace. Every GPU that loads this library holds the array until
// the process exits.
namespace fks {

constexpr size_t NOALLOC_BYTES = size_t(16) << 20;  // 16 MiB of scratch per device
constexpr int64_t NOALLOC_MAX_CELLS = 65536;        // largest grid (e.g. 256 x 256, 40^3)
constexpr int64_t NOALLOC_MAX_COARSE = 256;         // largest coarsest multigrid level
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];
// Device address of g_noalloc_scratch on each device. In host code the array's
// name is only a host-side stand-in, so the address is looked up once per device
// with cudaGetSymbolAddress and that pointer is what the kernels get.
static void* g_noalloc_addr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;

static cudaError_t noalloc_scratch(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[device] = p;
  }
  *out = g_noalloc_addr[device];
  return cudaSuccess;
}

}  // namespace fks

extern "C" fks_status fks_precond_apply_noalloc(fks_op* op, fks_c128 tau, const fks_c128* v, fks_c128* z, double eps,
                                                int max_cycles, int cycles, int precision, int32_t* out_cycles,
                                                double* out_pnorm, void* stream) {
  if (!op || !v || !z) { set_error("fks_precond_apply_noalloc: NULL argument"); return FKS_ERR_ARG; }
  if (op->csr) { set_error("fks_precond_apply_noalloc: grid operators only"); return FKS_ERR_ARG; }
  if (!finite_c(tau)) { set_error("fks_precond_apply_noalloc: tau has NaN/Inf"); return FKS_ERR_ARG; }
  if (!prec_ok(precision)) {
    set_error("fks_precond_apply_noalloc: bad precision");
    return FKS_ERR_ARG;
  }
  if (cycles < 0 && !(eps > 0)) { set_error("fks_precond_apply_noalloc: eps must be positive"); return FKS_ERR_ARG; }
  if (op->n > NOALLOC_MAX_CELLS) {
    set_error("fks_precond_apply_noalloc: the grid has more than 65536 cells, the limit of the fixed scratch array");
    return FKS_ERR_ARG;
  }
  if (op->levels.back().n > NOALLOC_MAX_COARSE) {
    set_error("fks_precond_apply_noalloc: the coarsest multigrid level has more than 256 cells");
    return FKS_ERR_ARG;
  }
  if (op->ctx->device < 0 || op->ctx->device >= NOALLOC_MAX_DEVICES) {
    set_error("fks_precond_apply_noalloc: device index beyond 63");
    return FKS_ERR_ARG;
  }
  if (!is_device_ptr(v) || !is_device_ptr(z)) {
    set_error("fks_precond_apply_noalloc: v and z must be device memory");
    return FKS_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  try {
    CK(cudaSetDevice(op->ctx->device));
    void* base = nullptr;
    CK(noalloc_scratch(op->ctx->device, &base));
    Solve S{};
    S.op = op;
    S.lane = &op->lane0;
    S.s = s;
    S.nslot = 1;
    S.n_f = 1;
    S.n_tau = 1;
    S.m = 1;
    S.sched_len = 1;
    S.precision = precision;
    S.n = op->n;
    S.eps = eps;
    S.max_cycles = max_cycles > 0 ? max_cycles : 50;
    S.replay = cycles >= 0;
    SlotState st_host{};
    S.st_host = &st_host;
    auto run = [&](auto tag) -> bool {
      using VT = decltype(tag);
      Arena probe;
      carve<VT>(S, probe, false);
      if (probe.off > NOALLOC_BYTES) return false;
      Arena A;
      A.base = (char*)base;  // never reserve(): the arena only carves the fixed array
      A.cap = NOALLOC_BYTES;
      carve<VT>(S, A, false);
      int64_t n = S.n;
      // v is copied into the fixed array first, so z may alias v (an in-place
      // call): the defects of later cycles read the copy, not z
      CK(cudaMemcpyAsync(S.V, v, sizeof(z64) * n, cudaMemcpyDeviceToDevice, s));
      // z = 0 when no cycle runs (a replayed count of 0, or v = 0 in the eps mode)
      CK(cudaMemsetAsync(z, 0, sizeof(z64) * n, s));
      CK(cudaMemcpyAsync(S.taus, &tau, sizeof(z64), cudaMemcpyHostToDevice, s));
      int32_t cyc = cycles;
      CK(cudaMemcpyAsync(S.rep_cyc, &cyc, sizeof(int32_t), cudaMemcpyHostToDevice, s));
      SlotState st0{};
      st0.active = 1;
      st0.k = 1;
      st0.tau = 0;
      CK(cudaMemcpyAsync(S.st, &st0, sizeof(SlotState), cudaMemcpyHostToDevice, s));
      setup_levels<VT>(S);
      inner_solve<VT>(S, S.V, n, (z64*)z, n);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(S.st_host, S.st, sizeof(SlotState), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (out_cycles) *out_cycles = S.st_host->cycles;
      if (out_pnorm) *out_pnorm = std::sqrt(S.st_host->pnorm2);
      return true;
    };
    bool fits = precision == FKS_PREC_FP64 ? run(double{}) : run(float{});
    if (!fits) {
      set_error("fks_precond_apply_noalloc: the scratch this grid needs exceeds the 16 MiB fixed array");
      return FKS_ERR_ARG;
    }
  } catch (CudaError& e) {
    set_error(std::string("fks_precond_apply_noalloc: ") + e.where + ": " + cudaGetErrorString(e.e));
    return FKS_ERR_CUDA;
  }
  return FKS_OK;
}

// ====================================================================== serving
// A request loop over the solver: worker threads, each with a lane (stream,
// stream-ordered workspace, graph), admit queued requests while the device
// memory budget allows; a worker merges queued requests that share the
// operator, the shifts and the options into one lockstep batch (each request's
// sources are slots of the batch). Batches on different lanes overlap on the
// device. Every slot runs its own kernels, so a request's result does not
// depend on what it was batched with.
namespace fks {

struct Request {
  uint64_t ticket = 0;
  fks_request req{};
  std::vector<int32_t> sched;
  std::vector<fks_c128> sigma, tau;
  int state = 0;  // 0 queued, 1 running, 2 done, 3 cancelled
  fks_status result = FKS_OK;
  double t_submit = 0, t_start = 0, t_end = 0;
  size_t est = 0;
  bool cancel = false;   // fks_server_cancel while running: stop at the next step boundary
  int sources_left = 0;  // sources not yet delivered
  int next_src = 0;      // sources admitted so far (a request's sources are admitted in order as slots free up)
};

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static bool compatible(const Request& a, const Request& b) {
  const fks_request &x = a.req, &y = b.req;
  if (x.op != y.op || x.n_f != y.n_f || x.n_tau != y.n_tau) return false;
  const fks_options &p = x.opt, &q = y.opt;
  if (p.tol != q.tol || p.m_max != q.m_max || p.variant != q.variant || p.precision != q.precision ||
      p.inner_tol != q.inner_tol || p.inner_max_cycles != q.inner_max_cycles || p.replay_mode || q.replay_mode ||
      std::max(p.inner_steps, 0) != std::max(q.inner_steps, 0) || p.assembly != q.assembly ||
      std::max(p.inner_relax, 0.0) != std::max(q.inner_relax, 0.0) ||
      a.sched != b.sched)
    return false;
  for (int j = 0; j < x.n_f; ++j)
    if (a.sigma[j].re != b.sigma[j].re || a.sigma[j].im != b.sigma[j].im) return false;
  for (int j = 0; j < x.n_tau; ++j)
    if (a.tau[j].re != b.tau[j].re || a.tau[j].im != b.tau[j].im) return false;
  return true;
}

}  // namespace fks

struct fks_server {
  fks_ctx* ctx = nullptr;
  size_t budget = 0, in_use = 0;
  int max_batch = 64;
  int join_slots = 16;           // spare slots a batch reserves for requests that join it later
  int steps_per_launch = 1;      // Arnoldi steps between admissions
  std::atomic<int64_t> launches{0};
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::deque<std::shared_ptr<fks::Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<fks::Request>> all;
  uint64_t next = 1;
  bool stop = false;
  std::vector<std::thread> workers;
  std::vector<std::unique_ptr<fks::Lane>> lanes;
  std::vector<cudaStream_t> streams;
};

namespace fks {

template <typename VT>
static size_t request_bytes(const fks_request& r, int n_rhs) {
  Solve S{};
  S.op = r.op;
  S.nslot = n_rhs;
  S.n_f = r.n_f;
  S.n_tau = r.n_tau;
  S.m = r.opt.m_max;
  S.sched_len = r.opt.sched_len;
  S.precision = r.opt.precision;
  S.n = r.op->n;
  S.batching = true;
  Arena probe;
  carve<VT>(S, probe, false);
  // one source's x_j and the tensor-core assembly's slices of one source
  // (sources are delivered one at a time)
  const int kmax = std::min(r.opt.m_max, TC_MAX_KP / 2);
  const size_t tc = r.opt.assembly == 0 && tc_supported(kmax, S.n) ? tc_ws_bytes(tc_layout(S.n, r.n_f, kmax, 1)) : 0;
  return probe.off + tc + sizeof(z64) * (size_t)S.n * r.n_f + 4096;
}

// Free run of `cnt` consecutive slots in `use`, or -1.
struct SlotUse {
  std::shared_ptr<Request> q;
  int r = 0;          // the request's source in this slot
  bool done = false;  // delivered
};

static int free_run(const std::vector<SlotUse>& use, int cnt) {
  int run = 0;
  for (int i = 0; i < (int)use.size(); ++i) {
    run = use[i].q ? 0 : run + 1;
    if (run == cnt) return i - cnt + 1;
  }
  return -1;
}

// One slot's outputs: x_j = Z y_j (tensor cores, or FP64 beyond their bound),
// the true residuals, and the copies into the request's own arrays for its
// source u.r. Each source is assembled and checked alone, exactly as fks_solve
// does it (its own step count decides the kernel), so its results do not depend
// on the batch it ran in.
template <typename VT>
static void deliver_slot(Solve& S, Lane* lane, int sl, const SlotUse& u, cudaStream_t s, int* tc_err) {
  const int64_t n = S.n;
  const int nf = S.n_f, m = S.m;
  const int k = S.st_host[sl].k;
  const int64_t vsZ = (int64_t)m * n;
  z64* Xs = S.X;  // the lane's one-source delivery buffer
  const fks_request& R = u.q->req;
  if (R.opt.assembly == 0 && k >= 1 && tc_supported(k, n)) {
    TcLayout T = tc_layout(n, nf, k, 1);
    const size_t need = tc_ws_bytes(T);
    lane->tcws.reserve(need + 256);
    {
      std::lock_guard<std::mutex> build_lock(g_build_mu);
      tc_prepare();
    }
    lane->prof.all_launches += launch_tc_assemble(T, S.st + sl, S.Z + (size_t)sl * vsZ, vsZ, S.Y + (size_t)sl * nf * m,
                                                  S.mj + (size_t)sl * nf, nf, m, Xs, n, 1, lane->tcws.base, tc_err, s);
  } else {
    launch_assemble(S.Z + (size_t)sl * vsZ, vsZ, S.Y + (size_t)sl * nf * m, S.mj + (size_t)sl * nf, nf, m, Xs, n, 1, s);
    lane->prof.all_launches += 1;
  }
  const fks_op* op = S.op;
  const int nb = op->csr ? csr_blocks(n) : tres_blocks(op->levels[0]);
  if (op->csr)
    launch_csr_true_residual(op->cd.view<double>(n), S.sigma, nf, S.b + (size_t)sl * n, Xs,
                             S.tpart + (size_t)sl * nf * nb, S.st + sl, S.tres + (size_t)sl * nf, 1, s);
  else
    launch_true_residual(op->levels[0], S.sigma, nf, S.b + (size_t)sl * n, Xs, S.tpart + (size_t)sl * nf * nb,
                         S.st + sl, S.tres + (size_t)sl * nf, 1, s);
  lane->prof.all_launches += 2;
  const size_t o = (size_t)u.r * nf, so = (size_t)sl * nf;
  if (R.X) copy_out(R.X + o * n, Xs, sizeof(z64) * n * nf, s);
  copy_out(R.res_est + o, S.est + so, sizeof(double) * nf, s);
  copy_out(R.res_bound + o, S.bnd + so, sizeof(double) * nf, s);
  if (R.res_true) copy_out(R.res_true + o, S.tres + so, sizeof(double) * nf, s);
  copy_out(R.m_j + o, S.mj + so, sizeof(int32_t) * nf, s);
  copy_out(R.shift_status + o, S.sst + so, sizeof(int32_t) * nf, s);
}

// Request status from its delivered shifts (after the copies completed).
static fks_status request_status(const Request& q) {
  fks_status rs = FKS_OK;
  for (int j = 0; j < q.req.n_f * q.req.n_rhs; ++j) {
    const int32_t v = q.req.shift_status[j];
    if (v == 1 || v == -1) rs = FKS_NOT_CONVERGED;
    else if (v == 2 && rs == FKS_OK) rs = FKS_BREAKDOWN_EXACT;
  }
  return rs;
}

static void finish_request(fks_server* sv, Request& q, fks_status st, int state = 2) {
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    q.result = st;
    q.state = state;
    q.t_end = now_s();
  }
  sv->done_cv.notify_all();
}

// A lane's continuous batch (iteration-level batching): `cap` slots, one
// source each, for requests compatible with `first` (same operator, shifts,
// taus and options). The step loop runs `steps_per_launch` Arnoldi steps per
// launch of its graph; after each launch the server's driver thread
//  - delivers every source that finished (assembly, true residual, copies into
//    the request's arrays: per-source output delivery) and frees its slot,
//  - stops the slots of cancelled or timed-out requests (k_stop_slots),
//  - admits queued compatible requests into free slots (their sources start at
//    step 1 while the others go on: every kernel works per slot, with its own
//    step, tau and inner-solve state),
// and launches the loop again. The batch ends when no slot is busy and no
// compatible request is queued.
struct BatchBase {
  virtual ~BatchBase() {}
  // setup, first launch; false if the batch already ended (its requests failed)
  virtual bool start() = 0;
  // after the last launch completed: deliveries, stops, admissions, next
  // launch; false when the batch has ended
  virtual bool step_done() = 0;
  cudaEvent_t ev = nullptr;
  size_t est = 0;
  int lane_id = 0;
};

template <typename VT>
struct Batch : BatchBase {
  fks_server* sv;
  Lane* lane;
  cudaStream_t s;
  std::shared_ptr<Request> first;
  int cap;
  Solve S{};
  fks_options o{};
  std::vector<SlotUse> use;
  std::vector<SlotState> sth;
  std::vector<int32_t> stop_h, cyc_h;
  struct Admit {
    int slot;
    std::shared_ptr<Request> q;
    int r;
  };
  std::vector<Admit> admit;

  // the request's next sources into free slots (in order); false if some stay
  // pending. Caller holds sv->mu or runs before the batch is visible.
  bool admit_sources(const std::shared_ptr<Request>& q) {
    for (int i = 0; i < cap && q->next_src < q->req.n_rhs; ++i) {
      if (use[i].q) continue;
      use[i] = SlotUse{q, q->next_src, false};
      admit.push_back({i, q, q->next_src});
      ++q->next_src;
    }
    return q->next_src >= q->req.n_rhs;
  }

  Batch(fks_server* sv_, int lane_, std::shared_ptr<Request> first_, int cap_)
      : sv(sv_), lane(sv_->lanes[lane_].get()), s(sv_->streams[lane_]), first(std::move(first_)), cap(cap_) {
    lane_id = lane_;
    use.resize(cap);
    sth.resize(cap);
    stop_h.assign(cap, 0);
  }
  ~Batch() override {
    if (ev) cudaEventDestroy(ev);
  }

  // every request still holding (or about to take) a slot ends with `st`
  void fail_all(fks_status st) {
    std::vector<std::shared_ptr<Request>> qs;
    for (auto& u : use)
      if (u.q && std::find(qs.begin(), qs.end(), u.q) == qs.end()) qs.push_back(u.q);
    for (auto& a : admit)
      if (std::find(qs.begin(), qs.end(), a.q) == qs.end()) qs.push_back(a.q);
    if (first && first->next_src < first->req.n_rhs &&
        std::find(qs.begin(), qs.end(), first) == qs.end())
      qs.push_back(first);
    {
      // sources of these requests still queued are dropped with them
      std::lock_guard<std::mutex> lk(sv->mu);
      for (auto& q : qs) {
        auto it = std::find(sv->queue.begin(), sv->queue.end(), q);
        if (it != sv->queue.end()) sv->queue.erase(it);
      }
    }
    for (auto& q : qs) finish_request(sv, *q, st);
    for (auto& u : use) u = SlotUse{};
    admit.clear();
  }
  void fail(const CudaError& e) {
    set_error(std::string("fks_server: ") + e.where + ": " + cudaGetErrorString(e.e));
    cudaGetLastError();
    fail_all(e.e == cudaErrorMemoryAllocation ? FKS_ERR_OOM : FKS_ERR_CUDA);
  }

  bool start() override {
    const fks_request& r0 = first->req;
    fks_op* op = r0.op;
    const int64_t n = op->n;
    o = r0.opt;
    o.tau_schedule = first->sched.data();
    S.op = op;
    S.lane = lane;
    S.s = s;
    S.nslot = cap;
    S.n_f = r0.n_f;
    S.n_tau = r0.n_tau;
    S.m = o.m_max;
    S.sched_len = o.sched_len;
    S.precision = o.precision;
    S.variant = o.variant;
    S.n = n;
    S.tol = o.tol;
    S.eps = o.inner_tol > 0 ? o.inner_tol : std::min(1e-6, o.tol / 100.0);
    S.max_cycles = o.inner_max_cycles > 0 ? o.inner_max_cycles : 50;
    S.replay = false;
    S.inner_steps = o.inner_steps > 0 ? o.inner_steps : (op->csr && op->amg.on ? 4 : 8);
    S.relax = o.inner_relax > 0 ? o.inner_relax : 0.0;
    S.batching = true;
    S.st_host = sth.data();
    admit_sources(first);
    try {
      std::string err = amg_prepare<VT>(S, first->tau.data());
      if (!err.empty()) {
        set_error("fks_server: " + err);
        fail_all(FKS_ERR_ARG);
        return false;
      }
      Arena probe;
      carve<VT>(S, probe, false);
      lane->ws.reserve(probe.off + 4096);
      carve<VT>(S, lane->ws, false);
      lane->xws.reserve(sizeof(z64) * (size_t)n * S.n_f + 256);
      S.X = (z64*)lane->xws.base;
      if (S.amg) CK(cudaMemcpyAsync(S.amg_tab, S.amg_table.data(), S.amg_table.size(), cudaMemcpyHostToDevice, s));
      copy_in(S.sigma, first->sigma.data(), sizeof(z64) * S.n_f, s);
      copy_in(S.taus, first->tau.data(), sizeof(z64) * S.n_tau, s);
      CK(cudaMemcpyAsync(S.sched, o.tau_schedule, sizeof(int32_t) * o.sched_len, cudaMemcpyHostToDevice, s));
      setup_levels<VT>(S);
      CK(cudaMemsetAsync(S.st, 0, sizeof(SlotState) * cap, s));  // every slot idle
      std::vector<double> key = {(double)(uintptr_t)lane->ws.base, (double)cap, (double)S.n_f, (double)S.n_tau,
                                 (double)S.m, (double)S.sched_len, (double)S.precision, (double)S.variant, 0.0, S.eps,
                                 S.tol, (double)S.max_cycles, (double)op->fuse_max[0], (double)op->fuse_max[1],
                                 (double)S.inner_steps, (double)op->tile16_max[0], (double)op->tile16_max[1], S.relax,
                                 (double)op->tail_max[0], (double)op->tail_max[1], (double)op->cluster_max[0],
                                 (double)op->cluster_max[1], (double)op->tile8_max[0], (double)op->tile8_max[1], 0.0,
                                 (double)(S.amg ? op->amg.gen : -1), (double)S.amg_L, 1.0};
      for (int pz = 0; pz < 2; ++pz)
        for (int l = 0; l < MAX_LEVELS; ++l) key.push_back((double)op->zchunk[pz][l]);
      key.push_back((double)op->coop_max[0]);
      key.push_back((double)op->coop_max[1]);
      key.push_back((double)pdl_flag());
      if (!lane->graph || lane->graph_key != key) {
        if (lane->graph) cudaGraphExecDestroy(lane->graph);
        lane->graph = nullptr;
        build_graph_any<VT>(S, lane);
        key.back() = (double)pdl_flag();
        lane->graph_key = key;
      }
      CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      launch();
      return true;
    } catch (CudaError& e) {
      fail(e);
      return false;
    }
  }

  // sources of newly admitted requests start (beta, v_1, shift bookkeeping),
  // then a few Arnoldi steps of every busy slot; `ev` marks the end
  void launch() {
    const int64_t n = S.n;
    const int n_f = S.n_f, m = S.m;
    const int nbn = norm_blocks(n);
    const int64_t vsV = (int64_t)(m + 1) * n;
    for (auto& a : admit) {
      const int a0 = a.slot, nr = 1;
      copy_in(S.b + (size_t)a0 * n, a.q->req.b + (size_t)a.r * n, sizeof(z64) * n, s);
      launch_norm2_partial(S.st + a0, 0, S.b + (size_t)a0 * n, n, n, S.npart + (size_t)a0 * nbn, nr, s);
      launch_start(S.st + a0, nr, S.npart + (size_t)a0 * nbn, nbn, n_f, s);
      launch_init_v1(S.st + a0, S.b + (size_t)a0 * n, n, S.V + (size_t)a0 * vsV, vsV, nr, s,
                     S.V32 ? S.V32 + (size_t)a0 * vsV : nullptr);
      launch_init_shifts(S.st + a0, n_f, m, S.sst + (size_t)a0 * n_f, S.mj + (size_t)a0 * n_f,
                         S.est + (size_t)a0 * n_f, S.bnd + (size_t)a0 * n_f, S.Y + (size_t)a0 * n_f * m,
                         S.alpha + (size_t)a0 * n_f, nr, s);
      CK(cudaMemsetAsync(S.pn + (size_t)a0 * m, 0, sizeof(double) * m * nr, s));
      CK(cudaMemsetAsync(S.cyc + (size_t)a0 * m, 0, sizeof(int32_t) * m * nr, s));
      CK(cudaMemsetAsync(S.H + (size_t)a0 * (m + 1) * m, 0, sizeof(z64) * (m + 1) * m * nr, s));
      CK(cudaMemsetAsync(S.taus_k + (size_t)a0 * m, 0, sizeof(z64) * m * nr, s));
      lane->prof.all_launches += 4;
    }
    admit.clear();
    const int32_t steps = sv->steps_per_launch;
    CK(cudaMemcpyAsync(S.budget, &steps, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CK(cudaGraphLaunch(lane->graph, s));
    CK(cudaEventRecord(ev, s));
  }

  bool step_done() override {
    try {
      const int m = S.m;
      CK(cudaMemcpyAsync(S.st_host, S.st, sizeof(SlotState) * cap, cudaMemcpyDeviceToHost, s));
      cyc_h.resize((size_t)cap * m);
      CK(cudaMemcpyAsync(cyc_h.data(), S.cyc, sizeof(int32_t) * cap * m, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      // launches: per step the outer section, per inner iteration (the most
      // cycles any busy slot ran in its step) the inner section
      int mx = 0;
      for (int i = 0; i < cap; ++i)
        if (use[i].q && S.st_host[i].k >= 1)
          mx = std::max(mx, cyc_h[(size_t)i * m + S.st_host[i].k - 1]);
      lane->prof.all_launches += (int64_t)lane->graph_outer + (int64_t)mx * lane->graph_inner;
      // deliver finished sources
      std::vector<std::shared_ptr<Request>> completed;
      CK(cudaMemsetAsync(S.tcerr, 0, sizeof(int), s));
      for (int i = 0; i < cap; ++i) {
        SlotUse& u = use[i];
        if (!u.q || S.st_host[i].active) continue;
        deliver_slot<VT>(S, lane, i, u, s, S.tcerr);
        if (--u.q->sources_left == 0) completed.push_back(u.q);
        u = SlotUse{};  // the slot is free for the next source at once
      }
      int tc_h = 0;
      CK(cudaMemcpyAsync(&tc_h, S.tcerr, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (tc_h) throw CudaError{cudaErrorLaunchFailure, "tensor-core assembly: a wait gave up after two seconds"};
      for (auto& q : completed) finish_request(sv, *q, request_status(*q));
      // cancellations and timeouts, then admissions
      std::vector<std::pair<std::shared_ptr<Request>, fks_status>> stopping;
      bool busy = false;
      {
        std::lock_guard<std::mutex> lk(sv->mu);
        const double t = now_s();
        for (auto& u : use) {
          if (!u.q) continue;
          Request& q = *u.q;
          const bool late = q.req.timeout_s > 0 && t - q.t_start > q.req.timeout_s;
          if ((q.cancel || late) &&
              std::find_if(stopping.begin(), stopping.end(), [&](auto& p) { return p.first == u.q; }) == stopping.end())
            stopping.push_back({u.q, q.cancel ? FKS_ERR_CANCELLED : FKS_ERR_TIMEOUT});
        }
        for (auto& sp : stopping) {
          for (int i = 0; i < cap; ++i)
            if (use[i].q == sp.first) {
              stop_h[i] = 1;
              use[i] = SlotUse{};
            }
          auto qi = std::find(sv->queue.begin(), sv->queue.end(), sp.first);  // its sources not yet admitted
          if (qi != sv->queue.end()) sv->queue.erase(qi);
        }
        if (!sv->stop)
          for (auto it = sv->queue.begin(); it != sv->queue.end();) {
            if (!compatible(*first, **it) || free_run(use, 1) < 0) {
              ++it;
              continue;
            }
            std::shared_ptr<Request> q = *it;
            if (q->state == 0) {
              q->state = 1;
              q->t_start = t;
              q->sources_left = q->req.n_rhs;
            }
            if (admit_sources(q)) it = sv->queue.erase(it);
            else ++it;
          }
        for (auto& u : use) busy = busy || u.q != nullptr;
      }
      if (!stopping.empty()) {
        CK(cudaMemcpyAsync(S.stopv, stop_h.data(), sizeof(int32_t) * cap, cudaMemcpyHostToDevice, s));
        launch_stop_slots(S.st, S.stopv, cap, s);
        CK(cudaStreamSynchronize(s));
        std::fill(stop_h.begin(), stop_h.end(), 0);
        for (auto& sp : stopping) finish_request(sv, *sp.first, sp.second, sp.second == FKS_ERR_CANCELLED ? 3 : 2);
      }
      if (!busy) return false;
      launch();
      return true;
    } catch (CudaError& e) {
      fail(e);
      return false;
    }
  }
};

// Slots of a new batch: the first request's sources plus join_slots spare
// ones, within max_batch and the free budget; at least one (a request with
// more sources than fit runs them in turn as slots free up).
template <typename VT>
static int batch_slots(fks_server* sv, const Request& q, size_t* bytes) {
  const int nr = q.req.n_rhs;
  int cap = std::max(1, std::min(nr + sv->join_slots, sv->max_batch));
  const size_t one = request_bytes<VT>(q.req, 1);
  const size_t per = std::max<size_t>(1, request_bytes<VT>(q.req, 2) - one);
  const size_t avail = sv->budget > sv->in_use ? sv->budget - sv->in_use : 0;
  while (cap > 1 && one + (size_t)(cap - 1) * per > avail) --cap;
  *bytes = request_bytes<VT>(q.req, cap);
  return cap;
}

// The server's driver: one host thread issues every CUDA call of the server
// (no two threads ever call the runtime for it), and the lanes overlap on the
// device through their own streams and graphs. It polls the lanes' launches,
// runs each finished launch's host work, and starts a batch on an idle lane
// for the first queued request that fits the budget (a request larger than the
// whole budget runs when nothing else holds any of it).
static void driver_loop(fks_server* sv) {
  cudaSetDevice(sv->ctx->device);
  const int nl = (int)sv->lanes.size();
  std::vector<std::unique_ptr<BatchBase>> run(nl);
  auto end_batch = [&](int i) {
    // the lane's workspaces go back to the stream-ordered pool, so that the
    // budget accounts for all the memory the server holds
    Lane* lane = sv->lanes[i].get();
    if (lane->graph) cudaGraphExecDestroy(lane->graph);
    lane->graph = nullptr;
    lane->graph_key.clear();
    lane->ws.release();
    lane->tcws.release();
    lane->xws.release();
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->in_use -= run[i]->est;
    }
    run[i].reset();
    sv->done_cv.notify_all();
  };
  while (true) {
    bool progress = false, running = false;
    for (int i = 0; i < nl; ++i) {
      if (!run[i]) continue;
      const cudaError_t q = cudaEventQuery(run[i]->ev);
      if (q == cudaErrorNotReady) {
        running = true;
        continue;
      }
      progress = true;
      const int64_t l0 = sv->lanes[i]->prof.all_launches;
      bool more = false;
      // (a failed launch makes step_done's first call fail, which ends the batch's requests)
      more = run[i]->step_done();
      sv->launches += sv->lanes[i]->prof.all_launches - l0;
      if (more) running = true;
      else end_batch(i);
    }
    for (int i = 0; i < nl; ++i) {
      if (run[i]) continue;
      std::shared_ptr<Request> first;
      size_t est = 0;
      int cap = 0;
      {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) break;
        auto it = sv->queue.begin();
        for (; it != sv->queue.end(); ++it)
          if ((*it)->est + sv->in_use <= sv->budget || sv->in_use == 0) break;
        if (it == sv->queue.end()) break;
        first = *it;
        cap = first->req.opt.precision == FKS_PREC_FP64 ? batch_slots<double>(sv, *first, &est)
                                                        : batch_slots<float>(sv, *first, &est);
        sv->in_use += est;
        if (first->state == 0) {
          first->state = 1;
          first->t_start = now_s();
          first->sources_left = first->req.n_rhs;
        }
        // the request leaves the queue once all its sources have slots
        if (first->req.n_rhs - first->next_src <= cap) sv->queue.erase(it);
        if (first->req.opt.precision == FKS_PREC_FP64) run[i].reset(new Batch<double>(sv, i, first, cap));
        else run[i].reset(new Batch<float>(sv, i, first, cap));
      }
      progress = true;
      run[i]->est = est;
      const int64_t l0 = sv->lanes[i]->prof.all_launches;
      const bool ok = run[i]->start();
      sv->launches += sv->lanes[i]->prof.all_launches - l0;
      if (ok) running = true;
      else end_batch(i);
    }
    std::unique_lock<std::mutex> lk(sv->mu);
    if (sv->stop && !running) return;
    if (!progress) {
      if (running) sv->cv.wait_for(lk, std::chrono::microseconds(50));
      else sv->cv.wait(lk, [&] { return sv->stop || !sv->queue.empty(); });
    }
  }
}

}  // namespace fks

extern "C" fks_status fks_server_create(fks_ctx* ctx, size_t mem_budget_bytes, int lanes, fks_server** out) {
  if (!out) { set_error("fks_server_create: out is NULL"); return FKS_ERR_ARG; }
  *out = nullptr;
  if (!ctx || lanes < 1 || lanes > 64 || mem_budget_bytes == 0) {
    set_error("fks_server_create: need a context, 1..64 lanes and a positive budget");
    return FKS_ERR_ARG;
  }
  fks_server* sv = new fks_server;
  sv->ctx = ctx;
  sv->budget = mem_budget_bytes;
  try {
    CK(cudaSetDevice(ctx->device));
    for (int i = 0; i < lanes; ++i) {
      cudaStream_t st;
      CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      sv->streams.push_back(st);
      sv->lanes.emplace_back(new Lane);
      sv->lanes.back()->ws.astream = st;
      sv->lanes.back()->tcws.astream = st;
      sv->lanes.back()->xws.astream = st;
    }
  } catch (CudaError& e) {
    for (auto st : sv->streams) cudaStreamDestroy(st);
    delete sv;
    set_error(std::string("fks_server_create: ") + cudaGetErrorString(e.e));
    return FKS_ERR_CUDA;
  }
  sv->workers.emplace_back(driver_loop, sv);
  *out = sv;
  return FKS_OK;
}

extern "C" fks_status fks_server_submit(fks_server* sv, const fks_request* r, uint64_t* ticket) {
  if (!sv || !r || !ticket) { set_error("fks_server_submit: NULL argument"); return FKS_ERR_ARG; }
  const fks_options& o = r->opt;
  if (!r->op || !r->b || !r->sigma || !r->tau || !r->res_est || !r->res_bound || !r->m_j ||
      !r->shift_status || r->n_rhs < 1 || r->n_f < 1 || r->n_tau < 1 || r->n_tau > MAX_TAU ||
      o.m_max < 1 || o.m_max > MAX_M || !(o.tol > 0) || o.sched_len < 1 || !o.tau_schedule || o.replay_mode ||
      !prec_ok(o.precision) || (r->op && r->op->csr && o.precision == FKS_PREC_MIXED_BF16) ||
      (o.variant != FKS_FGMRES && o.variant != FKS_FFOM) || o.inner_steps > 64 ||
      (o.assembly != 0 && o.assembly != 1) || !std::isfinite(o.inner_relax) || o.restart_len != 0) {
    set_error("fks_server_submit: bad request (restarted solves go through fks_solve)");
    return FKS_ERR_ARG;
  }
  for (int i = 0; i < o.sched_len; ++i)
    if (o.tau_schedule[i] < 0 || o.tau_schedule[i] >= r->n_tau) { set_error("fks_server_submit: bad schedule"); return FKS_ERR_ARG; }
  if (is_device_ptr(r->b) || (r->X && is_device_ptr(r->X))) { set_error("fks_server_submit: request arrays must be host memory"); return FKS_ERR_ARG; }
  if (!(r->timeout_s >= 0.0)) { set_error("fks_server_submit: timeout_s must be >= 0"); return FKS_ERR_ARG; }
  auto q = std::make_shared<Request>();
  q->req = *r;
  q->sched.assign(o.tau_schedule, o.tau_schedule + o.sched_len);
  q->sigma.assign(r->sigma, r->sigma + r->n_f);
  q->tau.assign(r->tau, r->tau + r->n_tau);
  for (auto& z : q->sigma) if (!finite_c(z)) { set_error("fks_server_submit: sigma has NaN/Inf"); return FKS_ERR_ARG; }
  for (auto& z : q->tau) if (!finite_c(z)) { set_error("fks_server_submit: tau has NaN/Inf"); return FKS_ERR_ARG; }
  if (!csr_diag_ok(r->op, q->tau.data(), r->n_tau)) { set_error("fks_server_submit: K + tau M has a zero diagonal entry"); return FKS_ERR_ARG; }
  // the least a batch for it needs: one source's slot (more sources run as slots free up)
  q->est = o.precision == FKS_PREC_FP64 ? request_bytes<double>(*r, 1) : request_bytes<float>(*r, 1);
  q->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    q->ticket = sv->next++;
    sv->all[q->ticket] = q;
    sv->queue.push_back(q);
  }
  sv->cv.notify_all();
  *ticket = q->ticket;
  return FKS_OK;
}

extern "C" fks_status fks_server_poll(fks_server* sv, uint64_t ticket, int* done, fks_status* result) {
  if (!sv || !done) { set_error("fks_server_poll: NULL argument"); return FKS_ERR_ARG; }
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) { set_error("fks_server_poll: unknown ticket"); return FKS_ERR_ARG; }
  *done = it->second->state >= 2;
  if (result) *result = it->second->state == 3 ? FKS_ERR_CANCELLED : it->second->result;
  if (result && !*done) *result = FKS_OK;
  return FKS_OK;
}

extern "C" fks_status fks_server_wait(fks_server* sv, uint64_t ticket, fks_status* result) {
  if (!sv) { set_error("fks_server_wait: NULL server"); return FKS_ERR_ARG; }
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) { set_error("fks_server_wait: unknown ticket"); return FKS_ERR_ARG; }
  auto q = it->second;
  sv->done_cv.wait(lk, [&] { return q->state >= 2; });
  if (result) *result = q->state == 3 ? FKS_ERR_CANCELLED : q->result;
  return FKS_OK;
}

extern "C" fks_status fks_server_cancel(fks_server* sv, uint64_t ticket) {
  if (!sv) { set_error("fks_server_cancel: NULL server"); return FKS_ERR_ARG; }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) { set_error("fks_server_cancel: unknown ticket"); return FKS_ERR_ARG; }
    auto q = it->second;
    if (q->state >= 2) { set_error("fks_server_cancel: the request already finished"); return FKS_ERR_ARG; }
    if (q->state == 1) {
      // running: its worker stops its sources at the next step boundary
      q->cancel = true;
      return FKS_OK;
    }
    for (auto jt = sv->queue.begin(); jt != sv->queue.end(); ++jt)
      if (*jt == q) {
        sv->queue.erase(jt);
        break;
      }
    q->state = 3;
    q->t_end = now_s();
  }
  sv->done_cv.notify_all();
  return FKS_OK;
}

extern "C" fks_status fks_server_times(fks_server* sv, uint64_t ticket, double* submit_s, double* start_s,
                                       double* end_s) {
  if (!sv) { set_error("fks_server_times: NULL server"); return FKS_ERR_ARG; }
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) { set_error("fks_server_times: unknown ticket"); return FKS_ERR_ARG; }
  if (submit_s) *submit_s = it->second->t_submit;
  if (start_s) *start_s = it->second->t_start;
  if (end_s) *end_s = it->second->t_end;
  return FKS_OK;
}

extern "C" fks_status fks_server_launches(fks_server* sv, int64_t* launches) {
  if (!sv || !launches) { set_error("fks_server_launches: NULL argument"); return FKS_ERR_ARG; }
  // the workers add each finished batch's launches
  *launches = sv->launches.load();
  return FKS_OK;
}

extern "C" void fks_debug_fail_allocs(int count) { g_fail_allocs.store(count > 0 ? count : 0); }

extern "C" void fks_server_destroy(fks_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  for (auto& t : sv->workers) t.join();
  cudaSetDevice(sv->ctx->device);
  for (size_t i = 0; i < sv->lanes.size(); ++i) {
    sv->lanes[i]->release();
    cudaStreamSynchronize(sv->streams[i]);
    cudaStreamDestroy(sv->streams[i]);
  }
  delete sv;
}
