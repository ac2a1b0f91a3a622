// Krylov kernels of the flexible shifted solver:
//  - start: beta = ||b||, v_1 = b / beta (Algorithm 3, REQUIRE line)
//  - classical Gram-Schmidt with one re-orthogonalisation (CGS2) of w = M z_k
//    against v_1..v_k, h_{k+1,k} = ||w||, v_{k+1} = w / h_{k+1,k} (Algorithm 3);
//    in exact arithmetic it gives the same H_bar as the modified Gram-Schmidt loop
//  - per-shift incremental complex Givens QR of H_bar(sigma_j; T_k) =
//    [I; 0] + H_bar_k (sigma_j I - T_k) (Eq. shiftedarnoldimod), the FGMRES residual
//    |g_{k+1}| and the inexact-solve bound of Eq. trueresidual; FFOM solves the
//    square system (Algorithm 4)
//  - assembly x_j = Z_{m_j} y_j and the true residual ||b - (K + sigma_j M) x_j||.
#include "krylov.cuh"
#include "stencil.cuh"

namespace fks {

constexpr int LIVE = -1;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Per-block partial sums of |x|^2 over a slot's vector (fixed order).
__global__ void k_norm2_partial(const SlotState* st, int need_active, const z64* __restrict__ x, int64_t vs,
                                int64_t n, double* __restrict__ partial) {
  int slot = blockIdx.y;
  if (need_active && !st[slot].active) return;
  __shared__ double red[32];
  double a = 0.0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
    a += abs2(x[slot * vs + c]);
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    partial[(int64_t)slot * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_start(SlotState* st, int nslot, const double* __restrict__ partial, int nblocks, int nf) {
  __shared__ double red[32];
  int slot = blockIdx.x;
  double s = 0.0;
  for (int q = threadIdx.x; q < nblocks; q += blockDim.x) s += partial[(int64_t)slot * nblocks + q];
  s = block_sum(s, red);
  if (threadIdx.x != 0) return;
  SlotState& t = st[slot];
  t.beta = sqrt(s);
  t.active = t.beta > 0.0 ? 1 : 0;
  t.live = t.active ? nf : 0;
  t.k = 0;
  t.tau = 0;
  t.cycles = 0;
  t.inner_done = 0;
  t.breakdown = 0;
  t.inner_capped = 0;
  t.vnorm2 = 0.0;
  t.pnorm2 = 0.0;
  t.w0norm2 = 0.0;
  t.rmax = 1.0;
  t.rmax_next = 0ull;
}

// v_1 = b / beta; shift bookkeeping reset (status LIVE, g_1 = beta, Y = 0).
__global__ void k_init_v1(const SlotState* st, const z64* __restrict__ b, int64_t n, z64* __restrict__ V,
                          int64_t vsV, z32* __restrict__ V32) {
  int slot = blockIdx.y;
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n) return;
  double beta = st[slot].beta;
  z64 v = beta > 0.0 ? (1.0 / beta) * b[slot * n + c] : mk(0.0, 0.0);
  V[slot * vsV + c] = v;
  if (V32) V32[slot * vsV + c] = cvt<float>(v);
}

__global__ void k_init_shifts(const SlotState* st, int nf, int m, int32_t* sst, int32_t* mj, double* est,
                              double* bnd, z64* Y, double* alpha) {
  int slot = blockIdx.y;
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nf) return;
  int64_t sj = (int64_t)slot * nf + j;
  bool act = st[slot].active;
  sst[sj] = act ? LIVE : 0;
  mj[sj] = 0;
  est[sj] = 0.0;
  bnd[sj] = 0.0;
  alpha[sj] = 0.0;
  for (int i = 0; i < m; ++i) Y[sj * m + i] = mk(0.0, 0.0);
}

// Start of the next step (k <- k + 1, 1-based): tau index from the schedule, record tau_k.
__global__ void k_step_begin(SlotState* st, int nslot, const int32_t* __restrict__ sched, int sched_len,
                             const z64* __restrict__ taus, z64* __restrict__ taus_k, int m) {
  int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= nslot) return;
  SlotState& s = st[slot];
  if (!s.active) return;
  int step = s.k + 1;
  s.k = step;
  s.tau = sched[(step - 1) % sched_len];
  taus_k[(int64_t)slot * m + step - 1] = taus[s.tau];
  s.inner_done = 0;
  s.cycles = 0;
}

// w = M z_k and partial sums of |w|^2 (scale of the breakdown test).
__global__ void k_mass(const SlotState* st, const double* __restrict__ mm, const z64* __restrict__ Z, int64_t vsZ,
                       z64* __restrict__ w, int64_t n, double* __restrict__ partial) {
  int slot = blockIdx.y;
  if (!st[slot].active) return;
  __shared__ double red[32];
  const z64* z = Z + slot * vsZ + (int64_t)(st[slot].k - 1) * n;
  double a = 0.0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    z64 v = mm[c] * z[c];
    w[slot * n + c] = v;
    a += abs2(v);
  }
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    partial[(int64_t)slot * gridDim.x + blockIdx.x] = s;
  }
}

// Partial h_i = sum_rows conj(V_i[row]) w[row] for columns i < k, over a
// block of MD_THREADS * MD_ROWS rows and a chunk of MD_COLS columns.
__global__ void __launch_bounds__(MD_THREADS) k_mdot(const SlotState* st, const z64* __restrict__ V, int64_t vsV,
                                                     const z64* __restrict__ w, int64_t n, z64* __restrict__ partial) {
  int slot = blockIdx.y;
  if (!st[slot].active) return;
  int k = st[slot].k;
  int c0 = blockIdx.z * MD_COLS;
  if (c0 >= k) return;
  int c1 = min(k, c0 + MD_COLS);
  __shared__ z64 red[MD_THREADS / 32][MD_COLS];
  int64_t row0 = (int64_t)blockIdx.x * MD_THREADS * MD_ROWS + threadIdx.x;
  z64 wr[MD_ROWS];
#pragma unroll
  for (int r = 0; r < MD_ROWS; ++r) {
    int64_t row = row0 + (int64_t)r * MD_THREADS;
    wr[r] = row < n ? w[slot * n + row] : mk(0.0, 0.0);
  }
  const z64* Vs = V + slot * vsV;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = c0; c < c1; ++c) {
    const z64* col = Vs + (int64_t)c * n;
    // acc += conj(v) w with four fused multiply-adds per row
    z64 acc = mk(0.0, 0.0);
#pragma unroll
    for (int r = 0; r < MD_ROWS; ++r) {
      int64_t row = row0 + (int64_t)r * MD_THREADS;
      if (row < n) {
        const z64 a = col[row], b = wr[r];
        acc.re = fmaT(a.re, b.re, fmaT(a.im, b.im, acc.re));
        acc.im = fmaT(a.re, b.im, fmaT(-a.im, b.re, acc.im));
      }
    }
    acc.re = warp_sum(acc.re);
    acc.im = warp_sum(acc.im);
    if (lane == 0) red[warp][c - c0] = acc;
  }
  __syncthreads();
  int t = threadIdx.x;
  if (t < c1 - c0) {
    z64 s = mk(0.0, 0.0);
    for (int q = 0; q < MD_THREADS / 32; ++q) s = s + red[q][t];
    partial[((int64_t)slot * gridDim.x + blockIdx.x) * MAX_M + c0 + t] = s;
  }
}

// The first CGS projection of the mixed-precision solve: the partial sums of
// h_i = v_i^* w as k_mdot forms them, from the complex64 copy of the basis and
// w rounded to complex64, accumulated in fp32 (written as complex128 partials,
// summed by k_hreduce). Its error (about 1e-7 ||w||) is removed by the second,
// complex128 projection; both updates w -= V h stay complex128, so the Arnoldi
// relation M z_k = V_{k+1} h holds to complex128 rounding with h = h1 + h2.
__global__ void __launch_bounds__(MD_THREADS) k_mdot32(const SlotState* st, const z32* __restrict__ V, int64_t vsV,
                                                       const z64* __restrict__ w, int64_t n,
                                                       z64* __restrict__ partial) {
  int slot = blockIdx.y;
  if (!st[slot].active) return;
  int k = st[slot].k;
  int c0 = blockIdx.z * MD_COLS;
  if (c0 >= k) return;
  int c1 = min(k, c0 + MD_COLS);
  __shared__ z32 red[MD_THREADS / 32][MD_COLS];
  int64_t row0 = (int64_t)blockIdx.x * MD_THREADS * MD_ROWS + threadIdx.x;
  z32 wr[MD_ROWS];
#pragma unroll
  for (int r = 0; r < MD_ROWS; ++r) {
    int64_t row = row0 + (int64_t)r * MD_THREADS;
    wr[r] = row < n ? cvt<float>(w[slot * n + row]) : mk(0.f, 0.f);
  }
  const z32* Vs = V + slot * vsV;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = c0; c < c1; ++c) {
    const z32* col = Vs + (int64_t)c * n;
    z32 acc = mk(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < MD_ROWS; ++r) {
      int64_t row = row0 + (int64_t)r * MD_THREADS;
      if (row < n) {
        const z32 a = col[row], b = wr[r];
        acc.re = fmaT(a.re, b.re, fmaT(a.im, b.im, acc.re));
        acc.im = fmaT(a.re, b.im, fmaT(-a.im, b.re, acc.im));
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      acc.re += __shfl_down_sync(0xffffffffu, acc.re, o);
      acc.im += __shfl_down_sync(0xffffffffu, acc.im, o);
    }
    if (lane == 0) red[warp][c - c0] = acc;
  }
  __syncthreads();
  int t = threadIdx.x;
  if (t < c1 - c0) {
    z32 s = mk(0.f, 0.f);
    for (int q = 0; q < MD_THREADS / 32; ++q) s = s + red[q][t];
    partial[((int64_t)slot * gridDim.x + blockIdx.x) * MAX_M + c0 + t] = cvt<double>(s);
  }
}

// h[i] = sum over row blocks of the partials (fixed order), i < k.
__global__ void k_hreduce(const SlotState* st, const z64* __restrict__ partial, int nblocks, z64* __restrict__ h,
                          int64_t hstride) {
  int slot = blockIdx.x;
  if (!st[slot].active) return;
  int k = st[slot].k;
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = w; i < k; i += nw) {
    z64 s = mk(0.0, 0.0);
    for (int q = lane; q < nblocks; q += 32) s = s + partial[((int64_t)slot * nblocks + q) * MAX_M + i];
    s.re = warp_sum(s.re);
    s.im = warp_sum(s.im);
    if (lane == 0) h[(int64_t)slot * hstride + i] = s;
  }
}

// w -= sum_{i<k} V_i h_i
__global__ void k_maxpy(const SlotState* st, const z64* __restrict__ V, int64_t vsV, const z64* __restrict__ h,
                        int64_t hstride, z64* __restrict__ w, int64_t n) {
  int slot = blockIdx.y;
  if (!st[slot].active) return;
  int k = st[slot].k;
  __shared__ z64 hs[MAX_M];
  for (int i = threadIdx.x; i < k; i += blockDim.x) hs[i] = h[(int64_t)slot * hstride + i];
  __syncthreads();
  int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= n) return;
  const z64* Vs = V + slot * vsV;
  z64 acc = w[slot * n + row];
  // acc -= v h with four fused multiply-adds per column
  for (int i = 0; i < k; ++i) {
    const z64 v = Vs[(int64_t)i * n + row], h = hs[i];
    acc.re = fmaT(-v.re, h.re, fmaT(v.im, h.im, acc.re));
    acc.im = fmaT(-v.re, h.im, fmaT(-v.im, h.re, acc.im));
  }
  w[slot * n + row] = acc;
}

// H[:, k-1] = h1 + h2, h_{k+1,k} = ||w||, breakdown test, ||p_k|| recorded.
__global__ void k_arnoldi_finish(SlotState* st, int nslot, const z64* __restrict__ h12, const double* __restrict__ wpart,
                                 const double* __restrict__ mpart, int nblocks, z64* __restrict__ H, int m,
                                 double* __restrict__ pn, int32_t* __restrict__ cyc, double breakdown_rtol) {
  int slot = blockIdx.x;
  SlotState& s = st[slot];
  if (!s.active) return;
  int k = s.k;
  z64* Hc = H + (int64_t)slot * (m + 1) * m + (int64_t)(k - 1) * (m + 1);
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    Hc[i] = h12[((int64_t)slot * 2 + 0) * MAX_M + i] + h12[((int64_t)slot * 2 + 1) * MAX_M + i];
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < nblocks; q += blockDim.x) {
    a += wpart[(int64_t)slot * nblocks + q];
    b += mpart[(int64_t)slot * nblocks + q];
  }
  __shared__ double red[32];
  a = block_sum(a, red);
  b = block_sum(b, red);
  if (threadIdx.x == 0) {
    double hn = sqrt(a);
    Hc[k] = mk(hn, 0.0);
    s.w0norm2 = b;
    s.breakdown = (hn <= breakdown_rtol * sqrt(b)) ? 1 : 0;
    pn[(int64_t)slot * m + k - 1] = sqrt(s.pnorm2);
    cyc[(int64_t)slot * m + k - 1] = s.cycles;
  }
}

// v_{k+1} = w / h_{k+1,k}
// v_{k+1} = w / h_{k+1,k}; with V32 also its complex64 copy (the first CGS
// projection of the mixed-precision solve reads it)
__global__ void k_new_v(const SlotState* st, const z64* __restrict__ w, int64_t n, const z64* __restrict__ H, int m,
                        z64* __restrict__ V, int64_t vsV, z32* __restrict__ V32) {
  int slot = blockIdx.y;
  const SlotState& s = st[slot];
  if (!s.active || s.breakdown) return;
  int k = s.k;
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n) return;
  double hn = H[(int64_t)slot * (m + 1) * m + (int64_t)(k - 1) * (m + 1) + k].re;
  const z64 v = (1.0 / hn) * w[slot * n + c];
  V[slot * vsV + (int64_t)k * n + c] = v;
  if (V32) V32[slot * vsV + (int64_t)k * n + c] = cvt<float>(v);
}

__device__ __forceinline__ double cabs(z64 a) { return hypot(a.re, a.im); }

// Per-shift least-squares update, one warp per (slot, shift).
__global__ void __launch_bounds__(GV_WARPS * 32) k_givens(SlotState* st, int nf, int m, const z64* __restrict__ sigma,
                                                          const z64* __restrict__ H, const z64* __restrict__ taus_k,
                                                          const double* __restrict__ pn, double tol, int variant,
                                                          const int32_t* __restrict__ replay_mj, z64* g, double* rc,
                                                          z64* rs, z64* R, z64* Y, int32_t* sst, int32_t* mj,
                                                          double* est_out, double* bnd_out, double* alpha_out,
                                                          const double* __restrict__ tol_shift, z64* coef_out) {
  __shared__ z64 col[GV_WARPS][MAX_M + 1];
  __shared__ z64 yv[GV_WARPS][MAX_M];
  __shared__ z64 rhs[GV_WARPS][MAX_M];
  __shared__ z64 dg[GV_WARPS][MAX_M];      // reciprocals of the diagonal of R (or of the square factor)
  __shared__ double rcs[GV_WARPS][MAX_M];  // this shift's stored rotations, staged
  __shared__ z64 rss[GV_WARPS][MAX_M];
  __shared__ z64 sc[GV_WARPS][2];   // pre (diagonal before the new rotation), g_k before it
  __shared__ double sd[GV_WARPS];   // residual estimate
  __shared__ double sal[GV_WARPS];  // Prop. 3's alpha at this step
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int slot = blockIdx.y;
  int j = blockIdx.x * GV_WARPS + warp;
  if (j >= nf) return;
  SlotState& s = st[slot];
  if (!s.active) return;
  int64_t sj = (int64_t)slot * nf + j;
  if (sst[sj] != LIVE) return;
  int k = s.k;
  double beta = s.beta;
  const z64* Hc = H + (int64_t)slot * (m + 1) * m + (int64_t)(k - 1) * (m + 1);
  z64 dsig = sigma[j] - taus_k[(int64_t)slot * m + k - 1];
  z64* gj = g + sj * (m + 1);
  double* rcj = rc + sj * m;
  z64* rsj = rs + sj * m;
  z64* Rj = R + sj * m * m;
  z64* cl = col[warp];
  // the new column of H_bar(sigma_j; T) and the stored rotations, loaded by all
  // lanes at once; lane 0 then runs the dependent chain from shared memory
  for (int i = lane; i <= k; i += 32) cl[i] = dsig * Hc[i];
  for (int i = lane; i + 1 < k; i += 32) {
    rcs[warp][i] = rcj[i];
    rss[warp][i] = rsj[i];
  }
  __syncwarp();
  z64* Rc = Rj + (int64_t)(k - 1) * m;
  if (lane == 0) {
    cl[k - 1] = cl[k - 1] + mk(1.0, 0.0);
    for (int i = 0; i + 1 < k; ++i) {
      z64 a = cl[i], b = cl[i + 1];
      double c = rcs[warp][i];
      z64 sn = rss[warp][i];
      cl[i] = c * a + sn * b;
      cl[i + 1] = c * b - conj(sn) * a;
    }
    z64 a = cl[k - 1], b = cl[k];
    double aa = cabs(a), bb = cabs(b);
    double c;
    z64 sn, r;
    if (bb == 0.0) {
      c = 1.0; sn = mk(0.0, 0.0); r = a;
    } else if (aa == 0.0) {
      c = 0.0; sn = (1.0 / bb) * conj(b); r = mk(bb, 0.0);
    } else {
      double nu = hypot(aa, bb);
      z64 ph = (1.0 / aa) * a;
      c = aa / nu;
      sn = (1.0 / nu) * (ph * conj(b));
      r = nu * ph;
    }
    rcj[k - 1] = c;
    rsj[k - 1] = sn;
    Rc[k - 1] = r;
    if (k == 1) gj[0] = mk(beta, 0.0);
    z64 gk = gj[k - 1];
    gj[k - 1] = c * gk;
    gj[k] = mk(0.0, 0.0) - conj(sn) * gk;
    sc[warp][0] = a;      // diagonal of the square (FFOM) factor
    sc[warp][1] = gk;
    sd[warp] = cabs(gj[k]);
    // Prop. 3: alpha = ||eta H_k(sigma; T)^{-*} e_k||, eta = h_{k+1,k}(sigma - tau_k) = b.
    // With H_k(sigma; T) = Q R (the rotations so far), the last row of its
    // inverse has norm 1 / |R_kk| = 1 / |a|: alpha = |b| / |a|, the tangent of
    // the new rotation.
    sal[warp] = aa > 0.0 ? bb / aa : (bb > 0.0 ? (double)INFINITY : 0.0);
  }
  __syncwarp();
  for (int i = lane; i + 1 < k; i += 32) Rc[i] = cl[i];  // the rotated column of R
  __syncwarp();
  bool brk = s.breakdown != 0;
  int rmj = replay_mj ? replay_mj[sj] : 0;
  double est = sd[warp];
  if (tol_shift) tol = tol_shift[sj];  // a restarted solve gives each shift its own tolerance
  bool need = variant == 1 || est <= tol * beta || brk || k == m || (replay_mj && k == rmj);
  if (!need) {
    // still iterating: its estimate enters the next step's relaxed tolerance
    if (lane == 0) atomicMax(&s.rmax_next, (unsigned long long)__double_as_longlong(est / beta));
    return;
  }
  // back substitution: R y = g (FGMRES) or the square factor (FFOM). The
  // diagonal is staged first and every column of R is loaded one step ahead,
  // so the dependent chain over i waits on arithmetic, not on memory.
  // the reciprocals of the diagonal are formed here, by all lanes at once, so
  // that the dependent chain below multiplies instead of dividing (an FP64
  // division is a long dependent sequence on this GPU)
  for (int i = lane; i < k; i += 32) {
    rhs[warp][i] = gj[i];
    const z64 d = (variant == 1 && i == k - 1) ? sc[warp][0] : Rj[(int64_t)i * m + i];
    const double t = 1.0 / abs2(d);
    dg[warp][i] = mk(d.re * t, -d.im * t);
  }
  __syncwarp();
  if (variant == 1 && lane == 0) rhs[warp][k - 1] = sc[warp][1];
  __syncwarp();
  constexpr int RPL = MAX_M / 32;  // rows per lane
  z64 colv[RPL], nextv[RPL];
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    const int l = lane + 32 * q;
    colv[q] = l < k - 1 ? Rj[(int64_t)(k - 1) * m + l] : mk(0.0, 0.0);
  }
  for (int i = k - 1; i >= 0; --i) {
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int l = lane + 32 * q;
      nextv[q] = (i > 0 && l < i - 1) ? Rj[(int64_t)(i - 1) * m + l] : mk(0.0, 0.0);
    }
    if (lane == 0) yv[warp][i] = rhs[warp][i] * dg[warp][i];
    __syncwarp();
    z64 yi = yv[warp][i];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int l = lane + 32 * q;
      if (l < i) rhs[warp][l] = rhs[warp][l] - colv[q] * yi;
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < RPL; ++q) colv[q] = nextv[q];
  }
  if (variant == 1) est = cabs(dsig) * Hc[k].re * cabs(yv[warp][k - 1]);
  double part = 0.0;
  for (int i = lane; i < k; i += 32) part += cabs(yv[warp][i]) * pn[(int64_t)slot * m + i];
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  double bound = est + part;
  bool conv = bound <= tol * beta;
  bool freeze = replay_mj ? (k == rmj || brk) : (conv || brk || k == m);
  if (!freeze) {
    if (lane == 0) atomicMax(&s.rmax_next, (unsigned long long)__double_as_longlong(est / beta));
    return;
  }
  for (int i = lane; i < m; i += 32) Y[sj * m + i] = i < k ? yv[warp][i] : mk(0.0, 0.0);
  if (lane == 0) {
    mj[sj] = k;
    alpha_out[sj] = sal[warp];
    // FFOM: the residual is c v_{k+1}, c = -(sigma - tau_k) h_{k+1,k} y_k (Eq. fomresidualsimplified)
    if (coef_out) coef_out[sj] = mk(0.0, 0.0) - (Hc[k].re * yv[warp][k - 1]) * dsig;
    sst[sj] = conv ? 0 : (brk ? 2 : 1);
    est_out[sj] = est / beta;
    bnd_out[sj] = bound / beta;
    atomicSub(&s.live, 1);
  }
}

// End of a step: a slot stops when every shift is frozen, at breakdown or at
// m_max. One block; with `use_cond` it sets the graph's outer loop condition
// to "some slot still active".
// End of a step: sources with no live shift, a breakdown or m steps stop. With
// `budget` (steps left in this launch of the step loop, set by the host) the
// loop also stops when it runs out, so that the host can admit new sources
// into free slots between launches (continuous batching).
__global__ void k_step_end(SlotState* st, int nslot, int m, int use_cond, cudaGraphConditionalHandle cond,
                           int* budget) {
  int any = 0;
  for (int slot = threadIdx.x; slot < nslot; slot += blockDim.x) {
    SlotState& s = st[slot];
    if (!s.active) continue;
    s.rmax = __longlong_as_double((long long)s.rmax_next);
    s.rmax_next = 0ull;
    if (s.live <= 0 || s.breakdown || s.k >= m) s.active = 0;
    any |= s.active;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    if (budget) {
      const int left = *budget - 1;
      *budget = left;
      if (left <= 0) any = 0;
    }
    if (use_cond) cudaGraphSetConditional(cond, any ? 1u : 0u);
  }
}

// Stop every source whose flag is set (stop[slot] != 0): it takes no further
// step (the server's cancellation and timeouts, between launches of the loop).
__global__ void k_stop_slots(SlotState* st, const int* __restrict__ stop, int nslot) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot < nslot && stop[slot]) st[slot].active = 0;
}

// X[:, j] = Z Y[:, j] for a tile of AS_J shifts (Y is zero beyond m_j).
__global__ void k_assemble(const z64* __restrict__ Z, int64_t vsZ, const z64* __restrict__ Y, const int32_t* __restrict__ mj,
                           int nf, int m, z64* __restrict__ X, int64_t n, const SlotState* st, int skip_k_le) {
  int slot = blockIdx.y;
  if (st && st[slot].k <= skip_k_le) return;  // assembled on the tensor cores
  int j0 = blockIdx.z * AS_J;
  __shared__ z64 ys[AS_J][MAX_M];
  __shared__ int kmax_s;
  if (threadIdx.x == 0) {
    int km = 0;
    for (int jj = 0; jj < AS_J && j0 + jj < nf; ++jj) km = max(km, mj[(int64_t)slot * nf + j0 + jj]);
    kmax_s = km;
  }
  __syncthreads();
  int kmax = kmax_s;
  for (int t = threadIdx.x; t < AS_J * kmax; t += blockDim.x) {
    int jj = t / kmax, i = t % kmax;
    ys[jj][i] = (j0 + jj < nf) ? Y[((int64_t)slot * nf + j0 + jj) * m + i] : mk(0.0, 0.0);
  }
  __syncthreads();
  int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= n) return;
  z64 acc[AS_J];
#pragma unroll
  for (int jj = 0; jj < AS_J; ++jj) acc[jj] = mk(0.0, 0.0);
  const z64* Zs = Z + slot * vsZ;
  for (int i = 0; i < kmax; ++i) {
    z64 zv = Zs[(int64_t)i * n + row];
#pragma unroll
    for (int jj = 0; jj < AS_J; ++jj) acc[jj] = acc[jj] + zv * ys[jj][i];
  }
#pragma unroll
  for (int jj = 0; jj < AS_J; ++jj)
    if (j0 + jj < nf) X[((int64_t)slot * nf + j0 + jj) * n + row] = acc[jj];
}

// Partial sums of |b - (K + sigma_j M) x_j|^2, grid (i blocks, row blocks, n_f * slots).
__global__ void k_tres_partial(LevelView<double> L, const z64* __restrict__ sigma, int nf, const z64* __restrict__ b,
                               const z64* __restrict__ X, double* __restrict__ partial) {
  int slot = blockIdx.z / nf, j = blockIdx.z - slot * nf;
  __shared__ double red[GX * GY / 32];
  double a = 0.0;
  const z64 sg = sigma[j];
  const z64* x = X + ((int64_t)slot * nf + j) * L.n;
  const int i = blockIdx.x * GX + threadIdx.x;
  const int rows = L.ny * L.nz;
#pragma unroll
  for (int q = 0; q < TRES_ROWS; ++q) {
    const int row = (blockIdx.y * TRES_ROWS + q) * GY + threadIdx.y;
    if (i >= L.nx || row >= rows) continue;
    const int k = row / L.ny;
    const Cell p{i, row - k * L.ny, k};
    const int c = row * L.nx + i;
    // b - (K + sigma M) x with the neighbour terms accumulated onto b
    const double d = L.kd ? L.kd[c] : fsum(faces_at(L, p));
    const double mc = L.mm[c];
    const z64 r = defect_at(L, p, c, mk(fmaT(sg.re, mc, d), mulT(sg.im, mc)), b[slot * L.n + c], x);
    a = fmaT(r.re, r.re, a);
    a = fmaT(r.im, r.im, a);
  }
  a = warp_sum(a);
  int tl = thread_linear();
  if ((tl & 31) == 0) red[tl >> 5] = a;
  __syncthreads();
  if (tl == 0) {
    double s = 0.0;
    for (int q = 0; q < GX * GY / 32; ++q) s += red[q];
    int nblk = gridDim.x * gridDim.y;
    partial[((int64_t)slot * nf + j) * nblk + block_linear()] = s;
  }
}

__global__ void k_tres_finish(const SlotState* st, const double* __restrict__ partial, int nblocks, int nf, int nslot,
                              double* __restrict__ out) {
  int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (t >= nf * nslot) return;
  int slot = t / nf;
  double s = 0.0;
  for (int q = lane; q < nblocks; q += 32) s += partial[(int64_t)t * nblocks + q];
  s = warp_sum(s);
  if (lane != 0) return;
  double beta = st[slot].beta;
  out[t] = beta > 0.0 ? sqrt(s) / beta : 0.0;
}

// --------------------------------------------------------------------- launchers
static inline unsigned nbk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

int norm_blocks(int64_t n) { return (int)std::min<int64_t>(nbk(n, 256), 1024); }

void launch_norm2_partial(const SlotState* st, int need_active, const z64* x, int64_t vs, int64_t n, double* partial,
                          int nslot, cudaStream_t s) {
  dim3 g(norm_blocks(n), nslot);
  k_norm2_partial<<<g, 256, 0, s>>>(st, need_active, x, vs, n, partial);
}
void launch_start(SlotState* st, int nslot, const double* partial, int nblocks, int nf, cudaStream_t s) {
  k_start<<<nslot, 512, 0, s>>>(st, nslot, partial, nblocks, nf);
}
void launch_init_v1(const SlotState* st, const z64* b, int64_t n, z64* V, int64_t vsV, int nslot, cudaStream_t s,
                    z32* V32) {
  dim3 g(nbk(n, 256), nslot);
  k_init_v1<<<g, 256, 0, s>>>(st, b, n, V, vsV, V32);
}
void launch_init_shifts(const SlotState* st, int nf, int m, int32_t* sst, int32_t* mj, double* est, double* bnd,
                        z64* Y, double* alpha, int nslot, cudaStream_t s) {
  dim3 g(nbk(nf, 64), nslot);
  k_init_shifts<<<g, 64, 0, s>>>(st, nf, m, sst, mj, est, bnd, Y, alpha);
}
void launch_step_begin(SlotState* st, int nslot, const int32_t* sched, int sched_len, const z64* taus, z64* taus_k,
                       int m, cudaStream_t s) {
  k_step_begin<<<nbk(nslot, 64), 64, 0, s>>>(st, nslot, sched, sched_len, taus, taus_k, m);
}
void launch_mass(const SlotState* st, const double* mm, const z64* Z, int64_t vsZ, z64* w, int64_t n, double* partial,
                 int nslot, cudaStream_t s) {
  dim3 g(norm_blocks(n), nslot);
  k_mass<<<g, 256, 0, s>>>(st, mm, Z, vsZ, w, n, partial);
}
int mdot_blocks(int64_t n) { return (int)nbk(n, MD_THREADS * MD_ROWS); }
void launch_mdot(const SlotState* st, const z64* V, int64_t vsV, const z64* w, int64_t n, z64* partial, int kmax,
                 int nslot, cudaStream_t s) {
  dim3 g(mdot_blocks(n), nslot, nbk(kmax, MD_COLS));
  k_mdot<<<g, MD_THREADS, 0, s>>>(st, V, vsV, w, n, partial);
}
void launch_mdot32(const SlotState* st, const z32* V, int64_t vsV, const z64* w, int64_t n, z64* partial, int kmax,
                   int nslot, cudaStream_t s) {
  dim3 g(mdot_blocks(n), nslot, nbk(kmax, MD_COLS));
  k_mdot32<<<g, MD_THREADS, 0, s>>>(st, V, vsV, w, n, partial);
}
void launch_hreduce(const SlotState* st, const z64* partial, int64_t n, z64* h, int64_t hstride, int nslot,
                    cudaStream_t s) {
  k_hreduce<<<nslot, 1024, 0, s>>>(st, partial, mdot_blocks(n), h, hstride);
}
void launch_maxpy(const SlotState* st, const z64* V, int64_t vsV, const z64* h, int64_t hstride, z64* w, int64_t n,
                  int nslot, cudaStream_t s) {
  dim3 g2(nbk(n, 256), nslot);
  k_maxpy<<<g2, 256, 0, s>>>(st, V, vsV, h, hstride, w, n);
}
void launch_arnoldi_finish(SlotState* st, int nslot, const z64* h12, const double* wpart, const double* mpart,
                           int nblocks, z64* H, int m, double* pn, int32_t* cyc, double rtol, cudaStream_t s) {
  k_arnoldi_finish<<<nslot, 512, 0, s>>>(st, nslot, h12, wpart, mpart, nblocks, H, m, pn, cyc, rtol);
}
void launch_new_v(const SlotState* st, const z64* w, int64_t n, const z64* H, int m, z64* V, int64_t vsV, int nslot,
                  cudaStream_t s, z32* V32) {
  dim3 g(nbk(n, 256), nslot);
  k_new_v<<<g, 256, 0, s>>>(st, w, n, H, m, V, vsV, V32);
}
void launch_givens(SlotState* st, int nf, int m, const z64* sigma, const z64* H, const z64* taus_k, const double* pn,
                   double tol, int variant, const int32_t* replay_mj, z64* g, double* rc, z64* rs, z64* R, z64* Y,
                   int32_t* sst, int32_t* mj, double* est, double* bnd, double* alpha, int nslot, cudaStream_t s,
                   const double* tol_shift, z64* coef) {
  dim3 gr(nbk(nf, GV_WARPS), nslot);
  k_givens<<<gr, GV_WARPS * 32, 0, s>>>(st, nf, m, sigma, H, taus_k, pn, tol, variant, replay_mj, g, rc, rs, R, Y, sst,
                                        mj, est, bnd, alpha, tol_shift, coef);
}
void launch_step_end(SlotState* st, int nslot, int m, int use_cond, cudaGraphConditionalHandle cond, cudaStream_t s,
                     int* budget) {
  k_step_end<<<1, 256, 0, s>>>(st, nslot, m, use_cond, cond, budget);
}
void launch_stop_slots(SlotState* st, const int* stop, int nslot, cudaStream_t s) {
  k_stop_slots<<<nbk(nslot, 64), 64, 0, s>>>(st, stop, nslot);
}
void launch_assemble(const z64* Z, int64_t vsZ, const z64* Y, const int32_t* mj, int nf, int m, z64* X, int64_t n,
                     int nslot, cudaStream_t s, const SlotState* st, int skip_k_le) {
  dim3 g(nbk(n, 256), nslot, nbk(nf, AS_J));
  k_assemble<<<g, 256, 0, s>>>(Z, vsZ, Y, mj, nf, m, X, n, st, skip_k_le);
}
int tres_blocks(const LevelHost& L) { return (int)(nbk(L.nx, GX) * nbk((int64_t)L.ny * L.nz, GY * TRES_ROWS)); }
void launch_true_residual(const LevelHost& L, const z64* sigma, int nf, const z64* b, const z64* X, double* partial,
                          const SlotState* st, double* out, int nslot, cudaStream_t s) {
  dim3 g(nbk(L.nx, GX), nbk((int64_t)L.ny * L.nz, GY * TRES_ROWS), nf * nslot);
  k_tres_partial<<<g, dim3(GX, GY), 0, s>>>(view<double>(L), sigma, nf, b, X, partial);
  launch_tres_finish(st, partial, tres_blocks(L), nf, nslot, out, s);
}
// X[idx[i]] += a[i] Xh[idx[i]] for the columns of a restart cycle (x_j += C_j d_j)
__global__ void k_axpy_cols(z64* __restrict__ X, const z64* __restrict__ Xh, const int32_t* __restrict__ idx,
                            const z64* __restrict__ a, int64_t n) {
  const int i = blockIdx.y;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  z64* x = X + (int64_t)idx[i] * n + c;
  *x = *x + a[i] * Xh[(int64_t)idx[i] * n + c];
}
void launch_axpy_cols(z64* X, const z64* Xh, const int32_t* idx, const z64* a, int ncols, int64_t n, cudaStream_t s) {
  k_axpy_cols<<<dim3(nbk(n, 256), ncols), 256, 0, s>>>(X, Xh, idx, a, n);
}
void launch_tres_finish(const SlotState* st, const double* partial, int nblocks, int nf, int nslot, double* out,
                        cudaStream_t s) {
  k_tres_finish<<<nbk((int64_t)nf * nslot, 8), 256, 0, s>>>(st, partial, nblocks, nf, nslot, out);
}

}  // namespace fks
