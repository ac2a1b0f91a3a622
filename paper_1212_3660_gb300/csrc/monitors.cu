// Prop. 1's Ritz values (Section 3, Eq. genritz): the eigenvalues theta of
// H_m(sigma; T_m) f = theta H_m f. Since H_m^{-1} H_m(sigma; T_m) = H_m^{-1} - T_m
// + sigma I, they are the eigenvalues of G = H_m^{-1} - T_m shifted by sigma;
// this file computes those of G, one warp per source, in three stages on a
// dense m x m copy in global scratch (m <= 128):
//   1. H_m^{-1} by Gauss-Jordan elimination with partial pivoting;
//   2. reduction of G to upper Hessenberg form by Householder reflections;
//   3. shifted QR iterations (Givens rotations, Wilkinson shift of the trailing
//      2 x 2 block, exceptional shifts after 10 stalled sweeps) with deflation
//      of negligible subdiagonal entries, for at most 60 m sweeps.
#include "monitors.cuh"

namespace fks {

namespace {

__device__ __forceinline__ double cab(z64 a) { return hypot(a.re, a.im); }

__device__ __forceinline__ z64 cdv(z64 a, z64 b) {
  // a / b by Smith's method
  if (fabs(b.re) >= fabs(b.im)) {
    const double r = b.im / b.re, d = b.re + b.im * r;
    return mk((a.re + a.im * r) / d, (a.im - a.re * r) / d);
  }
  const double r = b.re / b.im, d = b.re * r + b.im;
  return mk((a.re * r + a.im) / d, (a.im * r - a.re) / d);
}

__device__ __forceinline__ z64 csq(z64 a) {
  // principal square root
  const double m = cab(a);
  if (m == 0.0) return mk(0.0, 0.0);
  double re = sqrt(0.5 * (m + fabs(a.re)));
  double im = a.im / (2.0 * re);
  if (a.re < 0.0) {
    const double t = fabs(im);
    im = a.im < 0.0 ? -re : re;
    re = t;
  }
  return mk(re, im);
}

constexpr int RITZ_SWEEPS_PER_EIG = 60;

}  // namespace

// G: [n_rhs][m_max][m_max] scratch, Ginv the same; row-major per source.
__global__ void k_ritz(const z64* __restrict__ hbar, const z64* __restrict__ tau_k, const int32_t* __restrict__ steps,
                       int m_max, z64* __restrict__ Gs, z64* __restrict__ Ws, z64* __restrict__ theta,
                       int32_t* __restrict__ status) {
  const int r = blockIdx.x;
  const int lane = threadIdx.x;
  const int m = steps[r] < 0 ? 0 : (steps[r] > m_max ? m_max : steps[r]);
  z64* A = Gs + (int64_t)r * m_max * m_max;   // H_m, reduced in place
  z64* B = Ws + (int64_t)r * m_max * m_max;   // becomes H_m^{-1}, then G
  z64* th = theta + (int64_t)r * m_max;
  for (int i = lane; i < m_max; i += 32) th[i] = mk(0.0, 0.0);
  if (m <= 0) {
    if (lane == 0) status[r] = 0;
    return;
  }
  const z64* H = hbar + (int64_t)r * (m_max + 1) * m_max;  // column-major, leading dimension m_max + 1
  for (int q = lane; q < m * m; q += 32) {
    const int i = q / m, j = q - i * m;
    A[i * m + j] = H[(int64_t)j * (m_max + 1) + i];
    B[i * m + j] = mk(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncwarp();
  // ---- 1. Gauss-Jordan: [A | B] -> [I | A^{-1}]
  int singular = 0;
  for (int c = 0; c < m; ++c) {
    double best = -1.0;
    int piv = c;
    for (int i = c + lane; i < m; i += 32) {
      const double v = cab(A[i * m + c]);
      if (v > best) { best = v; piv = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_down_sync(0xffffffffu, best, o);
      const int op = __shfl_down_sync(0xffffffffu, piv, o);
      if (ob > best || (ob == best && op < piv)) { best = ob; piv = op; }
    }
    best = __shfl_sync(0xffffffffu, best, 0);
    piv = __shfl_sync(0xffffffffu, piv, 0);
    if (!(best > 0.0)) { singular = 1; break; }
    if (piv != c)
      for (int j = lane; j < m; j += 32) {
        z64 t = A[c * m + j]; A[c * m + j] = A[piv * m + j]; A[piv * m + j] = t;
        t = B[c * m + j]; B[c * m + j] = B[piv * m + j]; B[piv * m + j] = t;
      }
    __syncwarp();
    const z64 inv = cdv(mk(1.0, 0.0), A[c * m + c]);
    __syncwarp();
    for (int j = lane; j < m; j += 32) {
      A[c * m + j] = A[c * m + j] * inv;
      B[c * m + j] = B[c * m + j] * inv;
    }
    __syncwarp();
    for (int i = 0; i < m; ++i) {
      if (i == c) continue;
      const z64 f = A[i * m + c];
      __syncwarp();
      for (int j = lane; j < m; j += 32) {
        A[i * m + j] = A[i * m + j] - f * A[c * m + j];
        B[i * m + j] = B[i * m + j] - f * B[c * m + j];
      }
      __syncwarp();
    }
  }
  if (singular) {
    if (lane == 0) status[r] = 2;
    return;
  }
  // G = H_m^{-1} - T_m, kept in B
  for (int i = lane; i < m; i += 32) B[i * m + i] = B[i * m + i] - tau_k[(int64_t)r * m_max + i];
  __syncwarp();
  z64* G = B;
  z64* v = A;  // the inverse is done: A's storage holds a Householder vector
  // ---- 2. Householder reduction to upper Hessenberg form
  for (int c = 0; c + 2 < m; ++c) {
    double nrm2 = 0.0;
    for (int i = c + 1 + lane; i < m; i += 32) {
      const z64 x = G[i * m + c];
      nrm2 += x.re * x.re + x.im * x.im;
    }
    for (int o = 16; o > 0; o >>= 1) nrm2 += __shfl_xor_sync(0xffffffffu, nrm2, o);
    const z64 x0 = G[(c + 1) * m + c];
    const double nx = sqrt(nrm2), a0 = cab(x0);
    double tail = nrm2 - a0 * a0;
    if (!(tail > 1e-300 * nrm2) || nx == 0.0) continue;  // column already reduced
    const z64 ph = a0 > 0.0 ? mk(x0.re / a0, x0.im / a0) : mk(1.0, 0.0);
    const z64 alpha = mk(-nx * ph.re, -nx * ph.im);   // x - alpha e1 avoids cancellation
    for (int i = c + 1 + lane; i < m; i += 32) v[i] = G[i * m + c];
    __syncwarp();
    if (lane == 0) v[c + 1] = v[c + 1] - alpha;
    __syncwarp();
    double vn2 = 0.0;
    for (int i = c + 1 + lane; i < m; i += 32) vn2 += v[i].re * v[i].re + v[i].im * v[i].im;
    for (int o = 16; o > 0; o >>= 1) vn2 += __shfl_xor_sync(0xffffffffu, vn2, o);
    const double s = 2.0 / vn2;
    // G <- (I - s v v^*) G: rows c+1..m-1
    for (int j = lane; j < m; j += 32) {
      z64 w = mk(0.0, 0.0);
      for (int i = c + 1; i < m; ++i) w = w + conj(v[i]) * G[i * m + j];
      w = s * w;
      for (int i = c + 1; i < m; ++i) G[i * m + j] = G[i * m + j] - v[i] * w;
    }
    __syncwarp();
    // G <- G (I - s v v^*): columns c+1..m-1
    for (int i = lane; i < m; i += 32) {
      z64 w = mk(0.0, 0.0);
      for (int j = c + 1; j < m; ++j) w = w + G[i * m + j] * v[j];
      w = s * w;
      for (int j = c + 1; j < m; ++j) G[i * m + j] = G[i * m + j] - w * conj(v[j]);
    }
    __syncwarp();
    for (int i = c + 2 + lane; i < m; i += 32) G[i * m + c] = mk(0.0, 0.0);
    __syncwarp();
  }
  // ---- 3. shifted QR on the Hessenberg matrix (eigenvalues only: the
  // rotations are applied within the active window)
  int hi = m - 1, sweeps = 0, stalled = 0, fail = 0;
  const int max_sweeps = RITZ_SWEEPS_PER_EIG * m;
  z64* cs = v;  // rotation cosines at [i] (real part) and sines at [m_max + i]
  while (hi >= 0) {
    if (hi == 0) {
      if (lane == 0) th[0] = G[0];
      break;
    }
    // deflation: the largest lo with a negligible G[lo][lo-1]
    int lo = hi;
    while (lo > 0) {
      const double sub = cab(G[lo * m + lo - 1]);
      const double dia = cab(G[lo * m + lo]) + cab(G[(lo - 1) * m + lo - 1]);
      if (sub <= 1e-15 * dia || sub <= 1e-300) break;
      --lo;
    }
    if (lo == hi) {
      if (lane == 0) th[hi] = G[hi * m + hi];
      --hi;
      stalled = 0;
      continue;
    }
    if (++sweeps > max_sweeps) {
      fail = 1;
      for (int i = lane; i <= hi; i += 32) th[i] = G[i * m + i];
      break;
    }
    // shift: the eigenvalue of the trailing 2 x 2 block nearer its last diagonal entry
    const z64 a = G[(hi - 1) * m + hi - 1], b = G[(hi - 1) * m + hi], c2 = G[hi * m + hi - 1], d = G[hi * m + hi];
    z64 mu;
    if (++stalled % 11 == 10) {
      mu = d + mk(cab(c2), 0.0);  // exceptional shift
    } else {
      const z64 hf = mk(0.5 * (a.re - d.re), 0.5 * (a.im - d.im));
      const z64 disc = csq(hf * hf + b * c2);
      const z64 m1 = d + hf + disc, m2 = d + hf - disc;  // (a + d)/2 +- disc
      const z64 e1 = m1 - d, e2 = m2 - d;
      mu = cab(e1) <= cab(e2) ? m1 : m2;
    }
    for (int i = lo + lane; i <= hi; i += 32) G[i * m + i] = G[i * m + i] - mu;
    __syncwarp();
    // QR: rotations zeroing the subdiagonal of rows lo+1..hi
    for (int i = lo; i < hi; ++i) {
      const z64 x = G[i * m + i], y = G[(i + 1) * m + i];
      const double ax = cab(x), ay = cab(y);
      double cr;
      z64 sn;
      if (ay == 0.0) {
        cr = 1.0; sn = mk(0.0, 0.0);
      } else if (ax == 0.0) {
        cr = 0.0; sn = mk(y.re / ay, -y.im / ay);
      } else {
        const double nu = hypot(ax, ay);
        cr = ax / nu;
        const z64 ph = mk(x.re / ax, x.im / ax);
        sn = (1.0 / nu) * (ph * conj(y));   // rows: [c s; -conj(s) c] [x; y] = [nu ph; 0]
      }
      __syncwarp();
      for (int j = i + lane; j <= hi; j += 32) {
        const z64 p = G[i * m + j], q = G[(i + 1) * m + j];
        G[i * m + j] = cr * p + sn * q;
        G[(i + 1) * m + j] = cr * q - conj(sn) * p;
      }
      if (lane == 0) {
        cs[i] = mk(cr, 0.0);
        cs[m_max + i] = sn;
      }
      __syncwarp();
    }
    // RQ: the adjoint rotations on the columns
    for (int i = lo; i < hi; ++i) {
      const double cr = cs[i].re;
      const z64 sn = cs[m_max + i];
      const int top = i + 1;  // R is upper triangular: rows lo..i+1 of columns i, i+1
      for (int k = lo + lane; k <= top; k += 32) {
        const z64 p = G[k * m + i], q = G[k * m + i + 1];
        G[k * m + i] = cr * p + conj(sn) * q;
        G[k * m + i + 1] = cr * q - sn * p;
      }
      __syncwarp();
    }
    for (int i = lo + lane; i <= hi; i += 32) G[i * m + i] = G[i * m + i] + mu;
    __syncwarp();
  }
  if (lane == 0) status[r] = fail;
}

void launch_ritz(const z64* hbar, const z64* tau_k, const int32_t* steps, int n_rhs, int m_max, z64* scratch,
                 z64* theta, int32_t* status, cudaStream_t s) {
  z64* G = scratch;
  z64* W = scratch + (size_t)n_rhs * m_max * m_max;
  k_ritz<<<n_rhs, 32, 0, s>>>(hbar, tau_k, steps, m_max, G, W, theta, status);
}

}  // namespace fks
