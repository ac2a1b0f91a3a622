// General sparse operator (CSR) kernels: y = (K + s M) x on the union pattern
// of K and M, the complex128 defect / mass / true-residual kernels of the
// solver, and the BiCGSTAB cycle of the inner solve (s Jacobi-preconditioned
// BiCGSTAB steps on A e = f from e = 0; the paper's inner Krylov method,
// Section 6), all batched over sources on gridDim.y.
#include <cooperative_groups.h>

#include <atomic>

#include "amg.cuh"
#include "csr.cuh"
#include "krylov.cuh"

namespace cg = cooperative_groups;

namespace fks {

__device__ __forceinline__ bool csr_running(const SlotState* st, int slot) {
  return st == nullptr || (st[slot].active && !st[slot].inner_done);
}

template <typename T>
__device__ __forceinline__ cx<T> csr_row(const CsrView<T>& A, int64_t row, cx<T> s, const cx<T>* __restrict__ x) {
  cx<T> acc = mk(T(0), T(0));
  const int nq = A.len[row];
  for (int q = 0; q < nq; ++q) {
    const int64_t e = csr_at(A, row, q);
    cx<T> a = mk(fmaT(s.re, A.mv[e], A.kv[e]), mulT(s.im, A.mv[e]));
    acc = acc + a * x[A.col[e]];
  }
  return acc;
}

// y = (K + s M) x, s fixed or tau of the slot
template <typename T>
__global__ void k_csr_apply(CsrView<T> A, z64 sfix, const SlotState* st, const z64* taus, const cx<T>* __restrict__ x,
                            cx<T>* __restrict__ y, int64_t vs) {
  int slot = blockIdx.y;
  int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= A.n) return;
  z64 s = st ? taus[st[slot].tau] : sfix;
  y[slot * vs + row] = csr_row(A, row, cvt<T>(s), x + slot * vs);
}

// r = v - (K + tau M) z (complex128), f0 = r in the cycle precision, partial |r|^2, |v|^2
template <typename T>
__global__ void k_csr_defect(CsrView<double> A, const SlotState* st, const z64* taus, const z64* __restrict__ v,
                             int64_t vsv, const z64* __restrict__ z, int64_t vsz, int64_t col, int zero_z,
                             cx<T>* __restrict__ f0, int64_t vsf, double* __restrict__ partial) {
  int slot = blockIdx.y;
  if (!csr_running(st, slot)) return;
  __shared__ double red[32];
  int64_t off = (int64_t)(st[slot].k - 1) * col;
  double r2 = 0.0, v2 = 0.0;
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < A.n; row += (int64_t)gridDim.x * blockDim.x) {
    z64 vv = v[slot * vsv + off + row];
    z64 r = zero_z ? vv : vv - csr_row(A, row, taus[st[slot].tau], z + slot * vsz + off);
    f0[slot * vsf + row] = cvt<T>(r);
    r2 += abs2(r);
    v2 += abs2(vv);
  }
  r2 = block_sum(r2, red);
  v2 = block_sum(v2, red);
  if (threadIdx.x == 0) {
    partial[((int64_t)slot * gridDim.x + blockIdx.x) * 2 + 0] = r2;
    partial[((int64_t)slot * gridDim.x + blockIdx.x) * 2 + 1] = v2;
  }
}

// w = M z_k (complex128) and partial |w|^2
__global__ void k_csr_mass(CsrView<double> A, const SlotState* st, const z64* __restrict__ Z, int64_t vsZ,
                           z64* __restrict__ w, double* __restrict__ partial) {
  int slot = blockIdx.y;
  if (!st[slot].active) return;
  __shared__ double red[32];
  const z64* z = Z + slot * vsZ + (int64_t)(st[slot].k - 1) * A.n;
  double a = 0.0;
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < A.n; row += (int64_t)gridDim.x * blockDim.x) {
    z64 acc = mk(0.0, 0.0);
    for (int q = 0; q < A.len[row]; ++q) {
      const int64_t e = csr_at(A, row, q);
      acc = axpy(A.mv[e], z[A.col[e]], acc);
    }
    w[slot * A.n + row] = acc;
    a += abs2(acc);
  }
  a = block_sum(a, red);
  if (threadIdx.x == 0) partial[(int64_t)slot * gridDim.x + blockIdx.x] = a;
}

// partial |b - (K + sigma_j M) x_j|^2, grid (blocks, n_f * slots)
__global__ void k_csr_tres_partial(CsrView<double> A, const z64* __restrict__ sigma, int nf, const z64* __restrict__ b,
                                   const z64* __restrict__ X, double* __restrict__ partial) {
  int slot = blockIdx.y / nf, j = blockIdx.y - slot * nf;
  __shared__ double red[32];
  const z64* x = X + ((int64_t)slot * nf + j) * A.n;
  double a = 0.0;
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < A.n; row += (int64_t)gridDim.x * blockDim.x)
    a += abs2(b[slot * A.n + row] - csr_row(A, row, sigma[j], x));
  a = block_sum(a, red);
  if (threadIdx.x == 0) partial[((int64_t)slot * nf + j) * gridDim.x + blockIdx.x] = a;
}

// 1 / (K_ii + tau M_ii) for every distinct tau
template <typename T>
__global__ void k_csr_dinv(int64_t n, const double* __restrict__ dk, const double* __restrict__ dm,
                           const z64* __restrict__ taus, int ntau, cx<T>* __restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int q = 0; q < ntau; ++q) {
    z64 D = mk(dk[i] + taus[q].re * dm[i], taus[q].im * dm[i]);
    double den = abs2(D);
    out[(int64_t)q * n + i] = cvt<T>(mk(D.re / den, -D.im / den));
  }
}

// ------------------------------------------------------------------ BiCGSTAB cycle
// Vector stage kernels (cycle precision T); scalars per slot in complex128.
template <typename T>
__global__ void k_bcg_init(const SlotState* st, BcgVecs<T> V, int64_t n, BcgScal* sc) {
  int slot = blockIdx.y;
  if (!csr_running(st, slot)) return;
  int64_t o = slot * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    cx<T> f = V.f[o + i];
    V.r[o + i] = f;
    V.rh[o + i] = f;
    V.p[o + i] = mk(T(0), T(0));
    V.v[o + i] = mk(T(0), T(0));
    V.e[o + i] = mk(T(0), T(0));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    BcgScal& s = sc[slot];
    s.rho_old = mk(1.0, 0.0);
    s.alpha = mk(1.0, 0.0);
    s.omega = mk(1.0, 0.0);
    s.halt = 0;
    s.last = 0;
  }
}

// partial sums of <a, b> (and <c, c> when c != nullptr) in complex128
template <typename T>
__global__ void k_bcg_dot(const SlotState* st, const BcgScal* sc, const cx<T>* __restrict__ a,
                          const cx<T>* __restrict__ b, const cx<T>* __restrict__ c, int64_t n, double* partial) {
  int slot = blockIdx.y;
  if (!csr_running(st, slot) || sc[slot].halt) return;
  __shared__ double red[32];
  int64_t o = slot * n;
  double re = 0.0, im = 0.0, cc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    z64 x = cvt<double>(a[o + i]), y = cvt<double>(b[o + i]);
    z64 d = cdot(x, y);
    re += d.re;
    im += d.im;
    if (c) cc += abs2(cvt<double>(c[o + i]));
  }
  re = block_sum(re, red);
  im = block_sum(im, red);
  cc = block_sum(cc, red);
  if (threadIdx.x == 0) {
    double* p = partial + ((int64_t)slot * gridDim.x + blockIdx.x) * 3;
    p[0] = re;
    p[1] = im;
    p[2] = cc;
  }
}

__device__ __forceinline__ bool czero(z64 a) { return a.re == 0.0 && a.im == 0.0; }
__device__ __forceinline__ z64 cdivd(z64 a, z64 b) {
  double d = abs2(b);
  return mk((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}

// stage 0: rho, beta; stage 1: alpha; stage 2: omega. One block per slot.
__global__ void k_bcg_scalar(const SlotState* st, BcgScal* sc, const double* __restrict__ partial, int nblocks,
                             int stage) {
  int slot = blockIdx.x;
  if (!csr_running(st, slot) || sc[slot].halt) return;
  __shared__ double red[32];
  double re = 0.0, im = 0.0, cc = 0.0;
  for (int q = threadIdx.x; q < nblocks; q += blockDim.x) {
    const double* p = partial + ((int64_t)slot * nblocks + q) * 3;
    re += p[0];
    im += p[1];
    cc += p[2];
  }
  re = block_sum(re, red);
  im = block_sum(im, red);
  cc = block_sum(cc, red);
  if (threadIdx.x != 0) return;
  BcgScal& s = sc[slot];
  z64 d = mk(re, im);
  if (stage == 0) {
    if (czero(d) || czero(s.omega)) { s.halt = 1; return; }
    s.rho = d;
    s.beta = cdivd(d, s.rho_old) * cdivd(s.alpha, s.omega);
  } else if (stage == 1) {
    if (czero(d)) { s.halt = 1; return; }
    s.alpha = cdivd(s.rho, d);
  } else {
    if (cc == 0.0) { s.omega = mk(0.0, 0.0); s.last = 1; return; }
    s.omega = mk(d.re / cc, d.im / cc);
  }
}

// p = r + beta (p - omega v); ph = dinv p (Jacobi), or with an AMG table the
// V-cycle's first sweep x1 = omega_0 D_0^{-1} p (the V-cycle then computes ph)
template <typename T>
__global__ void k_bcg_p(const SlotState* st, const BcgScal* sc, BcgVecs<T> V, const cx<T>* __restrict__ dinv,
                        const AmgLevel<T>* tab, int L, cx<T>* __restrict__ x1, int64_t n) {
  int slot = blockIdx.y;
  if (!csr_running(st, slot) || sc[slot].halt) return;
  const cx<T>* D = dinv ? dinv + (int64_t)st[slot].tau * n : nullptr;
  const AmgLevel<T>* A0 = tab ? tab + st[slot].tau * L : nullptr;
  cx<T> beta = cvt<T>(sc[slot].beta), om = cvt<T>(sc[slot].omega);
  int64_t o = slot * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    cx<T> p = V.r[o + i] + beta * (V.p[o + i] - om * V.v[o + i]);
    V.p[o + i] = p;
    if (D) V.ph[o + i] = D[i] * p;
    if (A0) x1[o + i] = amg_first(*A0, i, p);
  }
}

// y = A x for the BiCGSTAB products (slot tau), cycle precision
template <typename T>
__global__ void k_bcg_spmv(CsrView<T> A, const SlotState* st, const BcgScal* sc, const z64* taus,
                           const cx<T>* __restrict__ x, cx<T>* __restrict__ y) {
  int slot = blockIdx.y;
  if (!csr_running(st, slot) || sc[slot].halt) return;
  cx<T> s = cvt<T>(taus[st[slot].tau]);
  int64_t o = slot * A.n;
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < A.n; row += (int64_t)gridDim.x * blockDim.x)
    y[o + row] = csr_row(A, row, s, x + o);
}

// s = r - alpha v; sh = dinv s, or the AMG first sweep x1 = omega_0 D_0^{-1} s
template <typename T>
__global__ void k_bcg_s(const SlotState* st, const BcgScal* sc, BcgVecs<T> V, const cx<T>* __restrict__ dinv,
                        const AmgLevel<T>* tab, int L, cx<T>* __restrict__ x1, int64_t n) {
  int slot = blockIdx.y;
  if (!csr_running(st, slot) || sc[slot].halt) return;
  const cx<T>* D = dinv ? dinv + (int64_t)st[slot].tau * n : nullptr;
  const AmgLevel<T>* A0 = tab ? tab + st[slot].tau * L : nullptr;
  cx<T> al = cvt<T>(sc[slot].alpha);
  int64_t o = slot * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    cx<T> s = V.r[o + i] - al * V.v[o + i];
    V.s[o + i] = s;
    if (D) V.sh[o + i] = D[i] * s;
    if (A0) x1[o + i] = amg_first(*A0, i, s);
  }
}

// e += alpha ph + omega sh; r = s - omega t; rho_old = rho (the last step of a
// halting iteration, <t,t> = 0, has omega = 0)
template <typename T>
__global__ void k_bcg_update(const SlotState* st, BcgScal* sc, BcgVecs<T> V, int64_t n) {
  int slot = blockIdx.y;
  if (!csr_running(st, slot) || sc[slot].halt) return;
  cx<T> al = cvt<T>(sc[slot].alpha), om = cvt<T>(sc[slot].omega);
  int64_t o = slot * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    V.e[o + i] = V.e[o + i] + al * V.ph[o + i] + om * V.sh[o + i];
    V.r[o + i] = V.s[o + i] - om * V.t[o + i];
  }
}

__global__ void k_bcg_close(const SlotState* st, BcgScal* sc, int nslot) {
  int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= nslot || !csr_running(st, slot) || sc[slot].halt) return;
  sc[slot].rho_old = sc[slot].rho;
  if (sc[slot].last) sc[slot].halt = 1;
}

// The whole cycle in one cooperative launch. Every block runs the arithmetic of
// the stage kernels above over the same grid-stride partition (gridDim.x =
// csr_blocks(n), 256 threads), with the dot products accumulated in the loops
// that produce their operands (same elements, same order), and derives the
// scalars itself from the block partials exactly as k_bcg_scalar does: the
// results are bitwise those of the stage kernels. Grid barriers replace the
// launches (five per step); every block passes every barrier.
// csr_row with the vector read through L2 (x was written by other blocks
// before the last grid barrier: no stale L1 or read-only-cache copy)
template <typename T>
__device__ __forceinline__ cx<T> ldcg_cx(const cx<T>* p) {
  if constexpr (sizeof(T) == 8) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return mk(v.x, v.y);
  } else {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return mk(v.x, v.y);
  }
}

template <typename T>
__device__ __forceinline__ cx<T> csr_row_cg(const CsrView<T>& A, int64_t row, cx<T> s, const cx<T>* x) {
  cx<T> acc = mk(T(0), T(0));
  const int nq = A.len[row];
  for (int q = 0; q < nq; ++q) {
    const int64_t e = csr_at(A, row, q);
    cx<T> a = mk(fmaT(s.re, A.mv[e], A.kv[e]), mulT(s.im, A.mv[e]));
    acc = acc + a * ldcg_cx(x + A.col[e]);
  }
  return acc;
}

__device__ __forceinline__ void bcg_partial(double re, double im, double cc, double* red, double* partial, int slot) {
  re = block_sum(re, red);
  im = block_sum(im, red);
  cc = block_sum(cc, red);
  if (threadIdx.x == 0) {
    double* p = partial + ((int64_t)slot * gridDim.x + blockIdx.x) * 3;
    p[0] = re;
    p[1] = im;
    p[2] = cc;
  }
}

// k_bcg_scalar in every block, on a block-local copy of the slot's scalars
__device__ __forceinline__ void bcg_scalar_local(BcgScal& s, const double* __restrict__ partial, int slot, int stage,
                                                 double* red) {
  const int nblocks = gridDim.x;
  double re = 0.0, im = 0.0, cc = 0.0;
  for (int q = threadIdx.x; q < nblocks; q += blockDim.x) {
    const double* p = partial + ((int64_t)slot * nblocks + q) * 3;
    re += __ldcg(p);
    im += __ldcg(p + 1);
    cc += __ldcg(p + 2);
  }
  re = block_sum(re, red);
  im = block_sum(im, red);
  cc = block_sum(cc, red);
  if (threadIdx.x == 0) {
    z64 d = mk(re, im);
    if (stage == 0) {
      if (czero(d) || czero(s.omega)) s.halt = 1;
      else {
        s.rho = d;
        s.beta = cdivd(d, s.rho_old) * cdivd(s.alpha, s.omega);
      }
    } else if (stage == 1) {
      if (czero(d)) s.halt = 1;
      else s.alpha = cdivd(s.rho, d);
    } else {
      if (cc == 0.0) { s.omega = mk(0.0, 0.0); s.last = 1; }
      else s.omega = mk(d.re / cc, d.im / cc);
    }
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256) k_bcg_cycle(CsrView<T> A, const SlotState* st, const z64* taus, BcgVecs<T> V,
                                                   const cx<T>* __restrict__ dinv, BcgScal* scg, double* partial,
                                                   int steps) {
  cg::grid_group grid = cg::this_grid();
  const int slot = blockIdx.y;
  const bool run = csr_running(st, slot);
  const int64_t n = A.n, o = slot * n;
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
  __shared__ double red[32];
  __shared__ BcgScal sc;
  const int tau = run ? st[slot].tau : 0;
  const cx<T>* D = dinv + (int64_t)tau * n;
  const cx<T> shift = cvt<T>(taus[tau]);
  if (threadIdx.x == 0) {
    sc.rho_old = mk(1.0, 0.0);
    sc.alpha = mk(1.0, 0.0);
    sc.omega = mk(1.0, 0.0);
    sc.halt = run ? 0 : 1;
    sc.last = 0;
  }
  __syncthreads();
  // k_bcg_init, then the first step's <rh, r>
  {
    double re = 0.0, im = 0.0;
    if (run)
      for (int64_t i = i0; i < n; i += stride) {
        const cx<T> f = V.f[o + i];
        V.r[o + i] = f;
        V.rh[o + i] = f;
        V.p[o + i] = mk(T(0), T(0));
        V.v[o + i] = mk(T(0), T(0));
        V.e[o + i] = mk(T(0), T(0));
        const z64 d = cdot(cvt<double>(f), cvt<double>(f));
        re += d.re;
        im += d.im;
      }
    if (run) bcg_partial(re, im, 0.0, red, partial, slot);
  }
  for (int it = 0; it < steps; ++it) {
    grid.sync();
    if (!sc.halt) bcg_scalar_local(sc, partial, slot, 0, red);
    if (!sc.halt) {   // k_bcg_p
      const cx<T> beta = cvt<T>(sc.beta), om = cvt<T>(sc.omega);
      for (int64_t i = i0; i < n; i += stride) {
        const cx<T> p = V.r[o + i] + beta * (V.p[o + i] - om * V.v[o + i]);
        V.p[o + i] = p;
        V.ph[o + i] = D[i] * p;
      }
    }
    grid.sync();
    if (!sc.halt) {   // k_bcg_spmv (v = A ph) and <rh, v>
      double re = 0.0, im = 0.0;
      for (int64_t row = i0; row < n; row += stride) {
        const cx<T> y = csr_row_cg(A, row, shift, V.ph + o);
        V.v[o + row] = y;
        const z64 d = cdot(cvt<double>(V.rh[o + row]), cvt<double>(y));
        re += d.re;
        im += d.im;
      }
      bcg_partial(re, im, 0.0, red, partial, slot);
    }
    grid.sync();
    if (!sc.halt) bcg_scalar_local(sc, partial, slot, 1, red);
    if (!sc.halt) {   // k_bcg_s
      const cx<T> al = cvt<T>(sc.alpha);
      for (int64_t i = i0; i < n; i += stride) {
        const cx<T> sv = V.r[o + i] - al * V.v[o + i];
        V.s[o + i] = sv;
        V.sh[o + i] = D[i] * sv;
      }
    }
    grid.sync();
    if (!sc.halt) {   // k_bcg_spmv (t = A sh) and <t, s>, <t, t>
      double re = 0.0, im = 0.0, cc = 0.0;
      for (int64_t row = i0; row < n; row += stride) {
        const cx<T> y = csr_row_cg(A, row, shift, V.sh + o);
        V.t[o + row] = y;
        const z64 ty = cvt<double>(y);
        const z64 d = cdot(ty, cvt<double>(V.s[o + row]));
        re += d.re;
        im += d.im;
        cc += abs2(ty);
      }
      bcg_partial(re, im, cc, red, partial, slot);
    }
    grid.sync();
    if (!sc.halt) bcg_scalar_local(sc, partial, slot, 2, red);
    if (!sc.halt) {   // k_bcg_update and k_bcg_close, then the next step's <rh, r>
      const cx<T> al = cvt<T>(sc.alpha), om = cvt<T>(sc.omega);
      double re = 0.0, im = 0.0;
      for (int64_t i = i0; i < n; i += stride) {
        V.e[o + i] = V.e[o + i] + al * V.ph[o + i] + om * V.sh[o + i];
        const cx<T> r = V.s[o + i] - om * V.t[o + i];
        V.r[o + i] = r;
        const z64 d = cdot(cvt<double>(V.rh[o + i]), cvt<double>(r));
        re += d.re;
        im += d.im;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        sc.rho_old = sc.rho;
        if (sc.last) sc.halt = 1;
      }
      bcg_partial(re, im, 0.0, red, partial, slot);   // block_sum synchronises the block first
    }
  }
  if (run && blockIdx.x == 0 && threadIdx.x == 0) scg[slot] = sc;
}

// V_0(f0) -> out0 inside a cooperative cycle: the phases of the stage kernels
// of launch_amg_vcycle (same rows, same per-row arithmetic, so the same bits)
// separated by grid barriers. Every block of the launch passes every barrier:
// the loop bounds are kernel arguments, the same in all blocks; `work` only
// decides whether a block computes its rows. The first sweep of level 0 is in
// R.x[0] (written with f0).
template <typename T>
__device__ void amg_vcycle_grid(const AmgRun<T>& R, const AmgLevel<T>* lv, bool work, int slot, const cx<T>* f0,
                                cx<T>* out0, cg::grid_group& grid) {
  const int L = R.L, nu = R.nu;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
  cx<T>* cur[AMG_MAX_LEVELS];
  cx<T>* oth[AMG_MAX_LEVELS];
  for (int l = 0; l + 1 < L; ++l) {
    const int64_t n = R.n[l], o = slot * n;
    const cx<T>* f = (l == 0 ? f0 : R.f[l]) + o;
    cur[l] = R.x[l];
    oth[l] = R.y[l];
    for (int k = 1; k < nu; ++k) {
      grid.sync();
      if (work)
        for (int64_t i = t0; i < n; i += stride) oth[l][o + i] = amg_sweep(lv[l], i, f, cur[l] + o);
      cx<T>* t = cur[l];
      cur[l] = oth[l];
      oth[l] = t;
    }
    grid.sync();
    if (work)
      for (int64_t i = t0; i < n; i += stride) R.r[l][o + i] = amg_resid(lv[l], i, f, cur[l] + o);
    grid.sync();
    if (work) {
      const int64_t nc = R.n[l + 1];
      for (int64_t a = t0; a < nc; a += stride) {
        const cx<T> v = amg_row(lv[l].rrp, lv[l].rci, lv[l].rv, a, R.r[l] + o);
        R.f[l + 1][slot * nc + a] = v;
        if (l + 2 < L) R.x[l + 1][slot * nc + a] = amg_first(lv[l + 1], a, v);
      }
    }
  }
  grid.sync();
  if (work) {
    const int64_t n = R.n[L - 1];
    const cx<T>* f = (L == 1 ? f0 : R.f[L - 1]) + slot * n;
    cx<T>* out = (L == 1 ? out0 : R.r[L - 1]) + slot * n;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); row < n; row += warps) {
      const cx<T> v = amg_coarse_row(lv[L - 1], row, f, lane);
      if (lane == 0) out[row] = v;
    }
  }
  for (int l = L - 2; l >= 0; --l) {
    const int64_t n = R.n[l], o = slot * n, nc = R.n[l + 1];
    const cx<T>* f = (l == 0 ? f0 : R.f[l]) + o;
    cx<T>* out = (l == 0 ? out0 : R.r[l]) + o;
    grid.sync();
    if (work)
      for (int64_t i = t0; i < n; i += stride)
        cur[l][o + i] = amg_ld(cur[l] + o + i) + amg_row(lv[l].prp, lv[l].pci, lv[l].pv, i, R.r[l + 1] + slot * nc);
    for (int k = 0; k < nu; ++k) {
      grid.sync();
      cx<T>* dst = k == nu - 1 ? out : oth[l] + o;
      if (work)
        for (int64_t i = t0; i < n; i += stride) dst[i] = amg_sweep(lv[l], i, f, cur[l] + o);
      if (k < nu - 1) {
        cx<T>* t = cur[l];
        cur[l] = oth[l];
        oth[l] = t;
      }
    }
  }
}

// The AMG-preconditioned cycle in one cooperative launch: k_bcg_cycle's phases
// with ph = V(p), sh = V(s) (amg_vcycle_grid) in place of the Jacobi products.
// Bitwise the stage kernels of launch_bcg_cycle_amg.
template <typename T>
__global__ void __launch_bounds__(256) k_bcg_cycle_amg(CsrView<T> A, const SlotState* st, const z64* taus,
                                                       BcgVecs<T> V, AmgRun<T> R, BcgScal* scg, double* partial,
                                                       int steps) {
  cg::grid_group grid = cg::this_grid();
  const int slot = blockIdx.y;
  const bool run = csr_running(st, slot);
  const int64_t n = A.n, o = slot * n;
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
  __shared__ double red[32];
  __shared__ BcgScal sc;
  const int tau = run ? st[slot].tau : 0;
  const AmgLevel<T>* lv = R.tab + tau * R.L;
  const cx<T> shift = cvt<T>(taus[tau]);
  cx<T>* x1 = R.x[0];
  if (threadIdx.x == 0) {
    sc.rho_old = mk(1.0, 0.0);
    sc.alpha = mk(1.0, 0.0);
    sc.omega = mk(1.0, 0.0);
    sc.halt = run ? 0 : 1;
    sc.last = 0;
  }
  __syncthreads();
  {   // k_bcg_init, then the first step's <rh, r>
    double re = 0.0, im = 0.0;
    if (run)
      for (int64_t i = i0; i < n; i += stride) {
        const cx<T> f = V.f[o + i];
        V.r[o + i] = f;
        V.rh[o + i] = f;
        V.p[o + i] = mk(T(0), T(0));
        V.v[o + i] = mk(T(0), T(0));
        V.e[o + i] = mk(T(0), T(0));
        const z64 d = cdot(cvt<double>(f), cvt<double>(f));
        re += d.re;
        im += d.im;
      }
    if (run) bcg_partial(re, im, 0.0, red, partial, slot);
  }
  for (int it = 0; it < steps; ++it) {
    grid.sync();
    if (!sc.halt) bcg_scalar_local(sc, partial, slot, 0, red);
    if (!sc.halt) {   // k_bcg_p with the first sweep
      const cx<T> beta = cvt<T>(sc.beta), om = cvt<T>(sc.omega);
      for (int64_t i = i0; i < n; i += stride) {
        const cx<T> p = V.r[o + i] + beta * (V.p[o + i] - om * V.v[o + i]);
        V.p[o + i] = p;
        x1[o + i] = amg_first(lv[0], i, p);
      }
    }
    amg_vcycle_grid(R, lv, !sc.halt, slot, V.p, V.ph, grid);
    grid.sync();
    if (!sc.halt) {   // v = A ph and <rh, v>
      double re = 0.0, im = 0.0;
      for (int64_t row = i0; row < n; row += stride) {
        const cx<T> y = csr_row_cg(A, row, shift, V.ph + o);
        V.v[o + row] = y;
        const z64 d = cdot(cvt<double>(V.rh[o + row]), cvt<double>(y));
        re += d.re;
        im += d.im;
      }
      bcg_partial(re, im, 0.0, red, partial, slot);
    }
    grid.sync();
    if (!sc.halt) bcg_scalar_local(sc, partial, slot, 1, red);
    if (!sc.halt) {   // k_bcg_s with the first sweep
      const cx<T> al = cvt<T>(sc.alpha);
      for (int64_t i = i0; i < n; i += stride) {
        const cx<T> sv = V.r[o + i] - al * V.v[o + i];
        V.s[o + i] = sv;
        x1[o + i] = amg_first(lv[0], i, sv);
      }
    }
    amg_vcycle_grid(R, lv, !sc.halt, slot, V.s, V.sh, grid);
    grid.sync();
    if (!sc.halt) {   // t = A sh and <t, s>, <t, t>
      double re = 0.0, im = 0.0, cc = 0.0;
      for (int64_t row = i0; row < n; row += stride) {
        const cx<T> y = csr_row_cg(A, row, shift, V.sh + o);
        V.t[o + row] = y;
        const z64 ty = cvt<double>(y);
        const z64 d = cdot(ty, cvt<double>(V.s[o + row]));
        re += d.re;
        im += d.im;
        cc += abs2(ty);
      }
      bcg_partial(re, im, cc, red, partial, slot);
    }
    grid.sync();
    if (!sc.halt) bcg_scalar_local(sc, partial, slot, 2, red);
    if (!sc.halt) {   // k_bcg_update and k_bcg_close, then the next step's <rh, r>
      const cx<T> al = cvt<T>(sc.alpha), om = cvt<T>(sc.omega);
      double re = 0.0, im = 0.0;
      for (int64_t i = i0; i < n; i += stride) {
        V.e[o + i] = V.e[o + i] + al * amg_ld(V.ph + o + i) + om * amg_ld(V.sh + o + i);
        const cx<T> r = V.s[o + i] - om * V.t[o + i];
        V.r[o + i] = r;
        const z64 d = cdot(cvt<double>(V.rh[o + i]), cvt<double>(r));
        re += d.re;
        im += d.im;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        sc.rho_old = sc.rho;
        if (sc.last) sc.halt = 1;
      }
      bcg_partial(re, im, 0.0, red, partial, slot);   // block_sum synchronises the block first
    }
  }
  if (run && blockIdx.x == 0 && threadIdx.x == 0) scg[slot] = sc;
}

// ------------------------------------------------------------------ launchers
static inline unsigned cnb(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }
int csr_blocks(int64_t n) { return (int)std::min<int64_t>(cnb(n, 256), 512); }

template <typename T>
void launch_csr_apply(const CsrView<T>& A, z64 sfix, const SlotState* st, const z64* taus, const cx<T>* x, cx<T>* y,
                      int64_t vs, int nslot, cudaStream_t s) {
  k_csr_apply<T><<<dim3(cnb(A.n, 256), nslot), 256, 0, s>>>(A, sfix, st, taus, x, y, vs);
}

template <typename T>
void launch_csr_defect(const CsrView<double>& A, const SlotState* st, const z64* taus, const z64* v, int64_t vsv,
                       const z64* z, int64_t vsz, int64_t col, int zero_z, cx<T>* f0, int64_t vsf, double* partial,
                       int nslot, cudaStream_t s) {
  k_csr_defect<T><<<dim3(csr_blocks(A.n), nslot), 256, 0, s>>>(A, st, taus, v, vsv, z, vsz, col, zero_z, f0, vsf,
                                                               partial);
}

// partial sums over norm_blocks(n) blocks, the layout the Arnoldi finish reads
void launch_csr_mass(const CsrView<double>& A, const SlotState* st, const z64* Z, int64_t vsZ, z64* w, double* partial,
                     int nslot, cudaStream_t s) {
  k_csr_mass<<<dim3(norm_blocks(A.n), nslot), 256, 0, s>>>(A, st, Z, vsZ, w, partial);
}

void launch_csr_true_residual(const CsrView<double>& A, const z64* sigma, int nf, const z64* b, const z64* X,
                              double* partial, const SlotState* st, double* out, int nslot, cudaStream_t s) {
  int nb = csr_blocks(A.n);
  k_csr_tres_partial<<<dim3(nb, nf * nslot), 256, 0, s>>>(A, sigma, nf, b, X, partial);
  launch_tres_finish(st, partial, nb, nf, nslot, out, s);
}

template <typename T>
void launch_csr_dinv(int64_t n, const double* dk, const double* dm, const z64* taus, int ntau, cx<T>* out,
                     cudaStream_t s) {
  k_csr_dinv<T><<<cnb(n, 256), 256, 0, s>>>(n, dk, dm, taus, ntau, out);
}

// Blocks of 256 threads of `kernel` that can be resident at once on the
// current device, cached per (kernel variant, device): operators on devices with
// different SM counts or occupancy each get their own figure. 0 = not yet known
// (the cache holds the count + 1).
constexpr int COOP_MAX_DEVICES = 64;
static std::atomic<int> g_coop_resident[4][COOP_MAX_DEVICES];

template <typename Kern>
static int coop_capacity(int which, Kern kernel) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= COOP_MAX_DEVICES) {
    cudaGetLastError();
    return 0;
  }
  int r = g_coop_resident[which][dev].load(std::memory_order_relaxed);
  if (r > 0) return r - 1;
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 256, 0) != cudaSuccess) {
    cudaGetLastError();
    per = 0;
  }
  g_coop_resident[which][dev].store(per * sms + 1, std::memory_order_relaxed);
  return per * sms;
}

// one cycle: `steps` BiCGSTAB steps from e = 0 on A e = f
template <typename T>
void launch_bcg_cycle(const CsrView<T>& A, const SlotState* st, const z64* taus, const BcgVecs<T>& V,
                      const cx<T>* dinv, BcgScal* sc, double* partial, int steps, int nslot, cudaStream_t s,
                      int* launches) {
  int nbk = csr_blocks(A.n);
  dim3 g(nbk, nslot);
  // one cooperative launch when every block of the batch can be resident
  const int res = coop_capacity(sizeof(T) == 8 ? 0 : 1, k_bcg_cycle<T>);
  if ((int64_t)nbk * nslot <= res) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_bcg_cycle<T>, A, st, taus, V, dinv, sc, partial, steps) == cudaSuccess) {
      if (launches) *launches += 1;
      return;
    }
    cudaGetLastError();  // not launched: the stage kernels below compute the same
  }
  k_bcg_init<T><<<g, 256, 0, s>>>(st, V, A.n, sc);
  int cnt = 1;
  for (int it = 0; it < steps; ++it) {
    k_bcg_dot<T><<<g, 256, 0, s>>>(st, sc, V.rh, V.r, nullptr, A.n, partial);
    k_bcg_scalar<<<nslot, 256, 0, s>>>(st, sc, partial, nbk, 0);
    k_bcg_p<T><<<g, 256, 0, s>>>(st, sc, V, dinv, nullptr, 0, nullptr, A.n);
    k_bcg_spmv<T><<<g, 256, 0, s>>>(A, st, sc, taus, V.ph, V.v);
    k_bcg_dot<T><<<g, 256, 0, s>>>(st, sc, V.rh, V.v, nullptr, A.n, partial);
    k_bcg_scalar<<<nslot, 256, 0, s>>>(st, sc, partial, nbk, 1);
    k_bcg_s<T><<<g, 256, 0, s>>>(st, sc, V, dinv, nullptr, 0, nullptr, A.n);
    k_bcg_spmv<T><<<g, 256, 0, s>>>(A, st, sc, taus, V.sh, V.t);
    k_bcg_dot<T><<<g, 256, 0, s>>>(st, sc, V.t, V.s, V.t, A.n, partial);
    k_bcg_scalar<<<nslot, 256, 0, s>>>(st, sc, partial, nbk, 2);
    k_bcg_update<T><<<g, 256, 0, s>>>(st, sc, V, A.n);
    k_bcg_close<<<cnb(nslot, 64), 64, 0, s>>>(st, sc, nslot);
    cnt += 12;
  }
  if (launches) *launches += cnt;
}

int g_bcg_amg_coop = 1;

// one cycle with the AMG V-cycle as the preconditioner: one cooperative launch
// when the batch's blocks can all be resident, else the stage kernels, with
// ph = V(p) and sh = V(s) in place of the Jacobi products
template <typename T>
void launch_bcg_cycle_amg(const CsrView<T>& A, const SlotState* st, const z64* taus, const BcgVecs<T>& V,
                          const AmgRun<T>& R, BcgScal* sc, double* partial, int steps, int nslot, cudaStream_t s,
                          int* launches) {
  int nbk = csr_blocks(A.n);
  dim3 g(nbk, nslot);
  // one cooperative launch when every block of the batch can be resident
  const int res = coop_capacity(sizeof(T) == 8 ? 2 : 3, k_bcg_cycle_amg<T>);
  if ((int64_t)nbk * nslot <= res && g_bcg_amg_coop) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_bcg_cycle_amg<T>, A, st, taus, V, R, sc, partial, steps) == cudaSuccess) {
      if (launches) *launches += 1;
      return;
    }
    cudaGetLastError();  // not launched: the stage kernels below compute the same
  }
  k_bcg_init<T><<<g, 256, 0, s>>>(st, V, A.n, sc);
  int cnt = 1;
  for (int it = 0; it < steps; ++it) {
    k_bcg_dot<T><<<g, 256, 0, s>>>(st, sc, V.rh, V.r, nullptr, A.n, partial);
    k_bcg_scalar<<<nslot, 256, 0, s>>>(st, sc, partial, nbk, 0);
    k_bcg_p<T><<<g, 256, 0, s>>>(st, sc, V, nullptr, R.tab, R.L, R.x[0], A.n);
    cnt += 3 + launch_amg_vcycle<T>(R, st, sc, V.p, V.ph, nslot, s);
    k_bcg_spmv<T><<<g, 256, 0, s>>>(A, st, sc, taus, V.ph, V.v);
    k_bcg_dot<T><<<g, 256, 0, s>>>(st, sc, V.rh, V.v, nullptr, A.n, partial);
    k_bcg_scalar<<<nslot, 256, 0, s>>>(st, sc, partial, nbk, 1);
    k_bcg_s<T><<<g, 256, 0, s>>>(st, sc, V, nullptr, R.tab, R.L, R.x[0], A.n);
    cnt += 4 + launch_amg_vcycle<T>(R, st, sc, V.s, V.sh, nslot, s);
    k_bcg_spmv<T><<<g, 256, 0, s>>>(A, st, sc, taus, V.sh, V.t);
    k_bcg_dot<T><<<g, 256, 0, s>>>(st, sc, V.t, V.s, V.t, A.n, partial);
    k_bcg_scalar<<<nslot, 256, 0, s>>>(st, sc, partial, nbk, 2);
    k_bcg_update<T><<<g, 256, 0, s>>>(st, sc, V, A.n);
    k_bcg_close<<<cnb(nslot, 64), 64, 0, s>>>(st, sc, nslot);
    cnt += 5;
  }
  if (launches) *launches += cnt;
}

#define CSR_INST(T)                                                                                              \
  template void launch_csr_apply<T>(const CsrView<T>&, z64, const SlotState*, const z64*, const cx<T>*, cx<T>*,  \
                                    int64_t, int, cudaStream_t);                                                 \
  template void launch_csr_defect<T>(const CsrView<double>&, const SlotState*, const z64*, const z64*, int64_t,  \
                                     const z64*, int64_t, int64_t, int, cx<T>*, int64_t, double*, int,           \
                                     cudaStream_t);                                                              \
  template void launch_csr_dinv<T>(int64_t, const double*, const double*, const z64*, int, cx<T>*, cudaStream_t); \
  template void launch_bcg_cycle<T>(const CsrView<T>&, const SlotState*, const z64*, const BcgVecs<T>&,           \
                                    const cx<T>*, BcgScal*, double*, int, int, cudaStream_t, int*);           \
  template void launch_bcg_cycle_amg<T>(const CsrView<T>&, const SlotState*, const z64*, const BcgVecs<T>&,       \
                                        const AmgRun<T>&, BcgScal*, double*, int, int, cudaStream_t, int*);

CSR_INST(double)
CSR_INST(float)

}  // namespace fks
