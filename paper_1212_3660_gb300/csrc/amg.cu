// Smoothed-aggregation AMG (Vanek, Mandel & Brezina 1996) for the BiCGSTAB
// preconditioner of a CSR operator's inner solve; Section 6 names PyAMG's
// smoothed aggregation with BiCGSTAB and no parameters. The choices made here:
//   strength graph   the pattern of A_l (every stored connection is strong);
//                    level 0 keeps the entries where K or M is nonzero, and the
//                    products below keep every entry they produce, so the
//                    pattern of A_{l+1} is that of |P|^T |A_l| |P| whatever tau is
//   aggregation      pass 1 (ascending nodes): a node with no aggregated
//                    neighbour founds an aggregate with all of its neighbours;
//                    pass 2: each remaining node joins the aggregate of its
//                    first (ascending) neighbour placed by pass 1
//   tentative T      B_0 = 1; T[i, a] = B[i] / ||B on a||, B_{l+1}[a] = ||B on a||
//   prolongator      P = (I - omega D^{-1} A) T, omega = 4 / (3 rho),
//                    rho = max_i sum_j |a_ij| / |a_ii| (Gershgorin)
//   coarse operator  A_{l+1} = P^T A P (plain transpose)
//   coarsest         n_l <= max_coarse, l = max_levels - 1, or no coarsening:
//                    dense inverse (Gauss-Jordan with partial pivoting)
//   V-cycle          nu damped-Jacobi sweeps from zero, residual, restriction
//                    by P^T, coarse correction by P, nu sweeps.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "amg.cuh"
#include "csr.cuh"

namespace fks {

// ================================================================== host setup
namespace {

struct hz {   // host complex128; plain formulas (std::complex multiplication adds NaN/Inf recovery)
  double re, im;
};
inline hz H(z64 a) { return {a.re, a.im}; }
inline z64 Z(hz a) { return mk(a.re, a.im); }
inline hz operator*(hz a, hz b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline hz operator+(hz a, hz b) { return {a.re + b.re, a.im + b.im}; }
inline hz operator-(hz a, hz b) { return {a.re - b.re, a.im - b.im}; }
inline hz scale(double s, hz a) { return {s * a.re, s * a.im}; }
inline double habs(hz a) { return std::hypot(a.re, a.im); }
inline hz hinv(hz a) {
  double d = a.re * a.re + a.im * a.im;
  return {a.re / d, -a.im / d};
}

// C = A B over the structural product: every product term makes an entry
AmgCsr spgemm(const AmgCsr& A, const AmgCsr& B) {
  AmgCsr C;
  C.n = A.n;
  C.m = B.m;
  C.rp.assign(A.n + 1, 0);
  std::vector<int64_t> pos(B.m, -1);
  std::vector<int32_t> cols;
  std::vector<hz> acc;
  std::vector<int> ord;
  for (int64_t i = 0; i < A.n; ++i) {
    cols.clear();
    acc.clear();
    for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
      const int32_t k = A.ci[q];
      const hz a = H(A.v[q]);
      for (int64_t t = B.rp[k]; t < B.rp[k + 1]; ++t) {
        const int32_t j = B.ci[t];
        const hz p = a * H(B.v[t]);
        if (pos[j] < 0) {
          pos[j] = (int64_t)cols.size();
          cols.push_back(j);
          acc.push_back(p);
        } else {
          acc[pos[j]] = acc[pos[j]] + p;
        }
      }
    }
    ord.resize(cols.size());
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return cols[a] < cols[b]; });
    for (int o : ord) {
      C.ci.push_back(cols[o]);
      C.v.push_back(Z(acc[o]));
      pos[cols[o]] = -1;
    }
    C.rp[i + 1] = (int64_t)C.ci.size();
  }
  return C;
}

AmgCsr transpose(const AmgCsr& A) {
  AmgCsr T;
  T.n = A.m;
  T.m = A.n;
  T.rp.assign(A.m + 1, 0);
  for (int32_t c : A.ci) T.rp[c + 1]++;
  for (int64_t j = 0; j < A.m; ++j) T.rp[j + 1] += T.rp[j];
  T.ci.resize(A.ci.size());
  T.v.resize(A.v.size());
  std::vector<int64_t> next(T.rp.begin(), T.rp.end() - 1);
  for (int64_t i = 0; i < A.n; ++i)   // ascending rows: the columns of T come out sorted
    for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
      int64_t d = next[A.ci[q]]++;
      T.ci[d] = (int32_t)i;
      T.v[d] = A.v[q];
    }
  return T;
}

// standard aggregation on the off-diagonal pattern; -1 if a node stays alone
// after pass 2 (cannot happen: a node skipped by pass 1 has a pass-1 neighbour)
int32_t aggregate(const AmgCsr& A, std::vector<int32_t>& agg) {
  const int64_t n = A.n;
  agg.assign(n, -1);
  std::vector<char> first(n, 0);
  int32_t na = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] != -1) continue;
    bool free = true;
    for (int64_t q = A.rp[i]; q < A.rp[i + 1] && free; ++q)
      if (A.ci[q] != i && agg[A.ci[q]] != -1) free = false;
    if (!free) continue;
    agg[i] = na;
    first[i] = 1;
    for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
      if (A.ci[q] != i) {
        agg[A.ci[q]] = na;
        first[A.ci[q]] = 1;
      }
    ++na;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] != -1) continue;
    for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
      if (A.ci[q] != i && first[A.ci[q]]) {
        agg[i] = agg[A.ci[q]];
        break;
      }
    if (agg[i] == -1) return -1;
  }
  return na;
}

// dense inverse by Gauss-Jordan elimination with partial pivoting; false if singular
bool dense_inverse(const AmgCsr& A, std::vector<z64>& out) {
  const int64_t n = A.n;
  std::vector<hz> a((size_t)n * n, hz{0, 0}), b((size_t)n * n, hz{0, 0});
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) a[(size_t)i * n + A.ci[q]] = a[(size_t)i * n + A.ci[q]] + H(A.v[q]);
    b[(size_t)i * n + i] = hz{1, 0};
  }
  for (int64_t c = 0; c < n; ++c) {
    int64_t p = c;
    double best = habs(a[(size_t)c * n + c]);
    for (int64_t r = c + 1; r < n; ++r)
      if (habs(a[(size_t)r * n + c]) > best) {
        best = habs(a[(size_t)r * n + c]);
        p = r;
      }
    if (!(best > 0.0) || !std::isfinite(best)) return false;
    if (p != c)
      for (int64_t j = 0; j < n; ++j) {
        std::swap(a[(size_t)p * n + j], a[(size_t)c * n + j]);
        std::swap(b[(size_t)p * n + j], b[(size_t)c * n + j]);
      }
    const hz piv = hinv(a[(size_t)c * n + c]);
    for (int64_t j = 0; j < n; ++j) {
      a[(size_t)c * n + j] = a[(size_t)c * n + j] * piv;
      b[(size_t)c * n + j] = b[(size_t)c * n + j] * piv;
    }
    for (int64_t r = 0; r < n; ++r) {
      if (r == c) continue;
      const hz f = a[(size_t)r * n + c];
      if (f.re == 0.0 && f.im == 0.0) continue;
      for (int64_t j = 0; j < n; ++j) {
        a[(size_t)r * n + j] = a[(size_t)r * n + j] - f * a[(size_t)c * n + j];
        b[(size_t)r * n + j] = b[(size_t)r * n + j] - f * b[(size_t)c * n + j];
      }
    }
  }
  out.resize((size_t)n * n);
  for (size_t q = 0; q < out.size(); ++q) out[q] = Z(b[q]);
  return true;
}

}  // namespace

std::string amg_build(const AmgCsr& A0, int max_levels, int64_t max_coarse, AmgAgg* ag, AmgHost* out) {
  const bool given = !ag->agg.empty();
  out->lv.clear();
  out->cinv.clear();
  AmgCsr A = A0;
  std::vector<double> B(A.n, 1.0);
  for (int l = 0;; ++l) {
    AmgHostLevel L;
    const int64_t n = A.n;
    L.dinv.resize(n);
    double rho = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      hz d{0, 0};
      double rs = 0.0;
      for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
        rs += habs(H(A.v[q]));
        if (A.ci[q] == i) d = H(A.v[q]);
      }
      if (d.re == 0.0 && d.im == 0.0) return "AMG: zero diagonal entry on level " + std::to_string(l);
      L.dinv[i] = Z(hinv(d));
      rho = std::max(rho, rs / habs(d));
    }
    if (!std::isfinite(rho)) return "AMG: non-finite entry on level " + std::to_string(l);
    L.omega = 4.0 / (3.0 * rho);
    bool last;
    int32_t na = 0;
    if (given) {
      last = l == (int)ag->agg.size();
      if (!last) na = ag->count[l];
    } else {
      last = n <= max_coarse || l == max_levels - 1;
      if (!last) {
        std::vector<int32_t> a;
        na = aggregate(A, a);
        if (na < 0) return "AMG: aggregation left a node unassigned";
        last = na >= n;
        if (!last) {
          ag->agg.push_back(std::move(a));
          ag->count.push_back(na);
        }
      }
    }
    if (last) {
      if (n > AMG_MAX_DENSE)
        return "AMG: the coarsest level has " + std::to_string(n) + " unknowns (at most 4096)";
      if (!dense_inverse(A, out->cinv)) return "AMG: the coarsest level is singular";
      L.A = std::move(A);
      out->lv.push_back(std::move(L));
      return "";
    }
    const std::vector<int32_t>& agg = ag->agg[l];
    if ((int64_t)agg.size() != n) return "AMG: aggregates do not match the level";
    // tentative prolongator and the next near-null-space vector
    std::vector<double> nrm(na, 0.0);
    for (int64_t i = 0; i < n; ++i) nrm[agg[i]] += B[i] * B[i];
    for (auto& v : nrm) v = std::sqrt(v);
    AmgCsr T;
    T.n = n;
    T.m = na;
    T.rp.resize(n + 1);
    T.ci.resize(n);
    T.v.resize(n);
    for (int64_t i = 0; i < n; ++i) {
      T.rp[i] = i;
      T.ci[i] = agg[i];
      T.v[i] = mk(B[i] / nrm[agg[i]], 0.0);
    }
    T.rp[n] = n;
    // P = T - omega D^{-1} (A T) on the pattern of A T (which holds T's: A has its diagonal)
    AmgCsr P = spgemm(A, T);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t q = P.rp[i]; q < P.rp[i + 1]; ++q) {
        const hz t = P.ci[q] == agg[i] ? hz{T.v[i].re, 0.0} : hz{0.0, 0.0};
        P.v[q] = Z(t - scale(L.omega, H(L.dinv[i]) * H(P.v[q])));
      }
    AmgCsr R = transpose(P);
    AmgCsr Ac = spgemm(R, spgemm(A, P));
    B.assign(nrm.begin(), nrm.end());
    L.A = std::move(A);
    L.P = std::move(P);
    L.R = std::move(R);
    out->lv.push_back(std::move(L));
    A = std::move(Ac);
  }
}

namespace {

cudaError_t upload_raw(std::vector<void*>& mem, const void* src, size_t bytes, void** out) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) return e;
  mem.push_back(p);
  *out = p;
  return bytes ? cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
}

template <typename I>
cudaError_t upload_idx(std::vector<void*>& mem, const std::vector<I>& h, const I** out) {
  void* p = nullptr;
  cudaError_t e = upload_raw(mem, h.data(), sizeof(I) * h.size(), &p);
  *out = (const I*)p;
  return e;
}

template <typename T>
cudaError_t upload_cx(std::vector<void*>& mem, const std::vector<z64>& h, const cx<T>** out) {
  std::vector<cx<T>> c(h.size());
  for (size_t i = 0; i < h.size(); ++i) c[i] = mk((T)h[i].re, (T)h[i].im);
  void* p = nullptr;
  cudaError_t e = upload_raw(mem, c.data(), sizeof(cx<T>) * c.size(), &p);
  *out = (const cx<T>*)p;
  return e;
}

}  // namespace

template <typename T>
cudaError_t amg_upload(const AmgHost& h, std::vector<void*>& mem, std::vector<AmgLevel<T>>& levels) {
  levels.clear();
  cudaError_t e = cudaSuccess;
  auto ck = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  for (size_t l = 0; l < h.lv.size() && e == cudaSuccess; ++l) {
    const AmgHostLevel& H0 = h.lv[l];
    AmgLevel<T> L{};
    L.n = H0.A.n;
    ck(upload_idx(mem, H0.A.rp, &L.arp));
    ck(upload_idx(mem, H0.A.ci, &L.aci));
    ck(upload_cx<T>(mem, H0.A.v, &L.av));
    ck(upload_cx<T>(mem, H0.dinv, &L.dinv));
    L.omega = (T)H0.omega;
    if (l + 1 < h.lv.size()) {
      L.nc = H0.P.m;
      ck(upload_idx(mem, H0.P.rp, &L.prp));
      ck(upload_idx(mem, H0.P.ci, &L.pci));
      ck(upload_cx<T>(mem, H0.P.v, &L.pv));
      ck(upload_idx(mem, H0.R.rp, &L.rrp));
      ck(upload_idx(mem, H0.R.ci, &L.rci));
      ck(upload_cx<T>(mem, H0.R.v, &L.rv));
    } else {
      L.nc = 0;
      ck(upload_cx<T>(mem, h.cinv, &L.cinv));
    }
    levels.push_back(L);
  }
  return e;
}

// ================================================================== kernels
namespace {

__device__ __forceinline__ bool amg_live(const SlotState* st, const BcgScal* sc, int slot) {
  return (st == nullptr || (st[slot].active && !st[slot].inner_done)) && (sc == nullptr || !sc[slot].halt);
}

template <typename T>
__device__ __forceinline__ const AmgLevel<T>& amg_level(const AmgLevel<T>* tab, const SlotState* st, int slot,
                                                        int L, int l) {
  return tab[(st ? st[slot].tau : 0) * L + l];
}

// xo = xi + omega D^{-1} (f - A xi)
template <typename T>
__global__ void k_amg_smooth(const AmgLevel<T>* tab, int L, int l, const SlotState* st, const BcgScal* sc,
                             const cx<T>* f, const cx<T>* xi, cx<T>* __restrict__ xo, int64_t n) {
  const int slot = blockIdx.y;
  if (!amg_live(st, sc, slot)) return;
  const AmgLevel<T>& A = amg_level(tab, st, slot, L, l);
  const int64_t o = slot * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    xo[o + i] = amg_sweep(A, i, f + o, xi + o);
}

// r = f - A x
template <typename T>
__global__ void k_amg_resid(const AmgLevel<T>* tab, int L, int l, const SlotState* st, const BcgScal* sc,
                            const cx<T>* f, const cx<T>* x, cx<T>* __restrict__ r, int64_t n) {
  const int slot = blockIdx.y;
  if (!amg_live(st, sc, slot)) return;
  const AmgLevel<T>& A = amg_level(tab, st, slot, L, l);
  const int64_t o = slot * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[o + i] = amg_resid(A, i, f + o, x + o);
}

// fc = P^T r on level l + 1, and there (unless it is the coarsest) the first
// sweep xc = omega D^{-1} fc
template <typename T>
__global__ void k_amg_restrict(const AmgLevel<T>* tab, int L, int l, const SlotState* st, const BcgScal* sc,
                               const cx<T>* r, cx<T>* __restrict__ fc, cx<T>* __restrict__ xc, int64_t n, int64_t nc) {
  const int slot = blockIdx.y;
  if (!amg_live(st, sc, slot)) return;
  const AmgLevel<T>& A = amg_level(tab, st, slot, L, l);
  const AmgLevel<T>& C = amg_level(tab, st, slot, L, l + 1);
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < nc; a += (int64_t)gridDim.x * blockDim.x) {
    const cx<T> v = amg_row(A.rrp, A.rci, A.rv, a, r + slot * n);
    fc[slot * nc + a] = v;
    if (l + 2 < L) xc[slot * nc + a] = amg_first(C, a, v);
  }
}

// x += P e (e: the next level's result)
template <typename T>
__global__ void k_amg_prolong(const AmgLevel<T>* tab, int L, int l, const SlotState* st, const BcgScal* sc,
                              cx<T>* __restrict__ x, const cx<T>* e, int64_t n, int64_t nc) {
  const int slot = blockIdx.y;
  if (!amg_live(st, sc, slot)) return;
  const AmgLevel<T>& A = amg_level(tab, st, slot, L, l);
  const int64_t o = slot * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[o + i] = amg_ld(x + o + i) + amg_row(A.prp, A.pci, A.pv, i, e + slot * nc);
}

// out = Cinv f on the coarsest level, one warp per row
template <typename T>
__global__ void k_amg_coarse(const AmgLevel<T>* tab, int L, const SlotState* st, const BcgScal* sc,
                             const cx<T>* f, cx<T>* __restrict__ out, int64_t n) {
  const int slot = blockIdx.y;
  if (!amg_live(st, sc, slot)) return;
  const AmgLevel<T>& A = amg_level(tab, st, slot, L, L - 1);
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); row < n; row += warps) {
    const cx<T> v = amg_coarse_row(A, row, f + slot * n, lane);
    if (lane == 0) out[slot * n + row] = v;
  }
}

inline unsigned amg_blocks(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 1024); }

}  // namespace

template <typename T>
int launch_amg_vcycle(const AmgRun<T>& R, const SlotState* st, const BcgScal* sc, const cx<T>* f0, cx<T>* out0,
                      int nslot, cudaStream_t s) {
  const int L = R.L, nu = R.nu;
  int cnt = 0;
  cx<T>* cur[AMG_MAX_LEVELS];
  cx<T>* oth[AMG_MAX_LEVELS];
  for (int l = 0; l + 1 < L; ++l) {
    const int64_t n = R.n[l];
    const dim3 g(amg_blocks(n), nslot);
    const cx<T>* f = l == 0 ? f0 : R.f[l];
    cur[l] = R.x[l];   // holds the first sweep (written with f)
    oth[l] = R.y[l];
    for (int k = 1; k < nu; ++k) {
      k_amg_smooth<T><<<g, 256, 0, s>>>(R.tab, L, l, st, sc, f, cur[l], oth[l], n);
      std::swap(cur[l], oth[l]);
      ++cnt;
    }
    k_amg_resid<T><<<g, 256, 0, s>>>(R.tab, L, l, st, sc, f, cur[l], R.r[l], n);
    k_amg_restrict<T><<<dim3(amg_blocks(R.n[l + 1]), nslot), 256, 0, s>>>(R.tab, L, l, st, sc, R.r[l], R.f[l + 1],
                                                                          R.x[l + 1], n, R.n[l + 1]);
    cnt += 2;
  }
  {
    const int64_t n = R.n[L - 1];
    const unsigned nb = (unsigned)std::min<int64_t>((n + 7) / 8, 1024);   // 8 warps per block
    k_amg_coarse<T><<<dim3(nb, nslot), 256, 0, s>>>(R.tab, L, st, sc, L == 1 ? f0 : R.f[L - 1],
                                                    L == 1 ? out0 : R.r[L - 1], n);
    ++cnt;
  }
  for (int l = L - 2; l >= 0; --l) {
    const int64_t n = R.n[l];
    const dim3 g(amg_blocks(n), nslot);
    const cx<T>* f = l == 0 ? f0 : R.f[l];
    cx<T>* out = l == 0 ? out0 : R.r[l];
    k_amg_prolong<T><<<g, 256, 0, s>>>(R.tab, L, l, st, sc, cur[l], R.r[l + 1], n, R.n[l + 1]);
    ++cnt;
    for (int k = 0; k < nu; ++k) {
      cx<T>* dst = k == nu - 1 ? out : oth[l];
      k_amg_smooth<T><<<g, 256, 0, s>>>(R.tab, L, l, st, sc, f, cur[l], dst, n);
      ++cnt;
      if (k < nu - 1) std::swap(cur[l], oth[l]);
    }
  }
  return cnt;
}

#define AMG_INST(T)                                                                                       \
  template cudaError_t amg_upload<T>(const AmgHost&, std::vector<void*>&, std::vector<AmgLevel<T>>&);     \
  template int launch_amg_vcycle<T>(const AmgRun<T>&, const SlotState*, const BcgScal*, const cx<T>*,     \
                                    cx<T>*, int, cudaStream_t);

AMG_INST(double)
AMG_INST(float)

}  // namespace fks
