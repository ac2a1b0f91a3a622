// Structured-grid kernels: operator coefficients, the shifted operator apply,
// and the geometric-multigrid pieces of the inexact inner solve (Section 4,
// Eq. zmmoditer): red-black Gauss-Seidel, residual + restriction,
// interpolation + correction, coarsest-level dense solve.
//
// Every vector kernel takes a batch of sources ("slots") on gridDim.y; vector
// arguments point at slot 0 and consecutive slots are `vs` elements apart.
#include <algorithm>

#include "grid.cuh"
#include "stencil.cuh"

namespace fks {

__device__ __forceinline__ bool slot_running(const SlotState* st, int slot) {
  return st == nullptr || (st[slot].active && !st[slot].inner_done);
}

// --------------------------------------------------------------------- setup
// Fine-level faces from cell conductivity (harmonic mean on interior faces,
// 2 K A / h on zero-head faces). One thread per face of each orientation.
__global__ void k_faces_from_cond(int nx, int ny, int nz, double hx, double hy, double hz, uint32_t mask,
                                  const double* __restrict__ cond, double* fx, double* fy, double* fz) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t nfx = (int64_t)(nx + 1) * ny * nz, nfy = (int64_t)nx * (ny + 1) * nz;
  int64_t nfz = nz > 1 ? (int64_t)nx * ny * (nz + 1) : 0;
  if (t < nfx) {
    int i = (int)(t % (nx + 1));
    int64_t row = t / (nx + 1);  // k*ny + j
    double g = (hy * hz) / hx;
    int64_t c = row * nx + i;
    double v;
    if (i == 0) v = (mask & 1u) ? 2.0 * cond[c] * g : 0.0;
    else if (i == nx) v = (mask & 2u) ? 2.0 * cond[c - 1] * g : 0.0;
    else { double a = cond[c - 1], b = cond[c]; v = g * (2.0 * a * b / (a + b)); }
    fx[t] = v;
    return;
  }
  t -= nfx;
  if (t < nfy) {
    int i = (int)(t % nx);
    int64_t q = t / nx;
    int j = (int)(q % (ny + 1));
    int k = (int)(q / (ny + 1));
    double g = (hx * hz) / hy;
    int64_t c = ((int64_t)k * ny + j) * nx + i;
    double v;
    if (j == 0) v = (mask & 4u) ? 2.0 * cond[c] * g : 0.0;
    else if (j == ny) v = (mask & 8u) ? 2.0 * cond[c - nx] * g : 0.0;
    else { double a = cond[c - nx], b = cond[c]; v = g * (2.0 * a * b / (a + b)); }
    fy[t] = v;
    return;
  }
  t -= nfy;
  if (t < nfz) {
    int64_t sxy = (int64_t)nx * ny;
    int64_t ij = t % sxy;
    int k = (int)(t / sxy);
    double g = (hx * hy) / hz;
    int64_t c = (int64_t)k * sxy + ij;
    double v;
    if (k == 0) v = (mask & 16u) ? 2.0 * cond[c] * g : 0.0;
    else if (k == nz) v = (mask & 32u) ? 2.0 * cond[c - sxy] * g : 0.0;
    else { double a = cond[c - sxy], b = cond[c]; v = g * (2.0 * a * b / (a + b)); }
    fz[t] = v;
  }
}

// Coarse faces: (sum of the fine faces on the coarse face) x the face's factor
// (fine over coarse centre distance across it: 1/2 on evenly halved axes, 1 on
// axes not coarsened; fac_x/y/z, one per coarse face index along the axis);
// coarse mass: sum of the children. One thread per coarse face / cell. On an
// odd (ragged) axis the last coarse cell has one child: its high face is that
// child's, and the sums skip children past the fine grid.
__global__ void k_coarsen(LevelView<double> F, int rx, int ry, int rz, int cx_, int cy, int cz, double* fx,
                          double* fy, double* fz, double* mm, const double* __restrict__ fac_x,
                          const double* __restrict__ fac_y, const double* __restrict__ fac_z) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t nfx = (int64_t)(cx_ + 1) * cy * cz, nfy = (int64_t)cx_ * (cy + 1) * cz;
  int64_t nfz = cz > 1 || F.nz > 1 ? (int64_t)cx_ * cy * (cz + 1) : 0;
  int64_t ncell = (int64_t)cx_ * cy * cz;
  if (t < nfx) {
    int I = (int)(t % (cx_ + 1));
    int64_t q = t / (cx_ + 1);
    int J = (int)(q % cy), K = (int)(q / cy);
    double s = 0.0;
    const int64_t fi = min(rx * I, F.nx);
    for (int c = 0; c < rz; ++c)
      for (int b = 0; b < ry; ++b) {
        if (rz * K + c >= F.nz || ry * J + b >= F.ny) continue;
        int64_t row = (int64_t)(rz * K + c) * F.ny + (ry * J + b);
        s += F.fx[row * (F.nx + 1) + fi];
      }
    fx[t] = s * fac_x[I];
    return;
  }
  t -= nfx;
  if (t < nfy) {
    int I = (int)(t % cx_);
    int64_t q = t / cx_;
    int J = (int)(q % (cy + 1)), K = (int)(q / (cy + 1));
    double s = 0.0;
    const int64_t fj = min(ry * J, F.ny);
    for (int c = 0; c < rz; ++c)
      for (int a = 0; a < rx; ++a) {
        if (rz * K + c >= F.nz || rx * I + a >= F.nx) continue;
        s += F.fy[((int64_t)(rz * K + c) * (F.ny + 1) + fj) * F.nx + (rx * I + a)];
      }
    fy[t] = s * fac_y[J];
    return;
  }
  t -= nfy;
  if (t < nfz) {
    int64_t sxy = (int64_t)cx_ * cy;
    int64_t ij = t % sxy;
    int K = (int)(t / sxy);
    int I = (int)(ij % cx_), J = (int)(ij / cx_);
    double s = 0.0;
    const int64_t fk = min(rz * K, F.nz);
    for (int b = 0; b < ry; ++b)
      for (int a = 0; a < rx; ++a) {
        if (ry * J + b >= F.ny || rx * I + a >= F.nx) continue;
        s += F.fz[(fk * F.ny + (ry * J + b)) * F.nx + (rx * I + a)];
      }
    fz[t] = s * fac_z[K];
    return;
  }
  t -= nfz;
  if (t < ncell) {
    int I = (int)(t % cx_);
    int64_t q = t / cx_;
    int J = (int)(q % cy), K = (int)(q / cy);
    double s = 0.0;
    for (int c = 0; c < rz; ++c)
      for (int b = 0; b < ry; ++b)
        for (int a = 0; a < rx; ++a) {
          if (rz * K + c >= F.nz || ry * J + b >= F.ny || rx * I + a >= F.nx) continue;
          s += F.mm[((int64_t)(rz * K + c) * F.ny + (ry * J + b)) * F.nx + (rx * I + a)];
        }
    mm[t] = s;
  }
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) b[t] = (float)a[t];
}

// The bf16-smoother option's coefficients: a rounded to bf16 (nearest) and the
// same value as fp32 (exact).
__global__ void k_round_bf16(const double* __restrict__ a, __nv_bfloat16* __restrict__ b, float* __restrict__ r,
                             int64_t n) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const __nv_bfloat16 v = __double2bfloat16(a[t]);
  b[t] = v;
  r[t] = __bfloat162float(v);
}

// 1 / (K_cc + tau M_cc) per cell for every distinct tau, computed in fp64.
// (C: the coefficients' storage; the bf16-smoother option computes from the
// bf16-rounded values held as fp32)
template <typename T, typename C>
__global__ void k_invd(LevelView<double, C> L, const z64* __restrict__ taus, int ntau, cx<T>* __restrict__ out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  Cell p = cell_of(c, L.nx, L.ny);
  Faces<double> f = faces_at(L, p);
  double d = fsum(f), m = ldc<double>(L.mm, c);
  for (int q = 0; q < ntau; ++q) {
    z64 D = mk(d + taus[q].re * m, taus[q].im * m);
    double den = abs2(D);
    out[(int64_t)q * L.n + c] = cvt<T>(mk(D.re / den, -D.im / den));
  }
}

// Dense coarsest-level matrix K + tau M (row-major, n x n) for every tau.
template <typename C>
__global__ void k_coarse_dense(LevelView<double, C> L, const z64* __restrict__ taus, int ntau, z64* __restrict__ A) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  Cell p = cell_of(c, L.nx, L.ny);
  Faces<double> f = faces_at(L, p);
  double d = fsum(f), m = ldc<double>(L.mm, c);
  int64_t n = L.n, sxy = (int64_t)L.nx * L.ny;
  for (int q = 0; q < ntau; ++q) {
    z64* row = A + (int64_t)q * n * n + c * n;
    for (int64_t l = 0; l < n; ++l) row[l] = mk(0.0, 0.0);
    row[c] = mk(d + taus[q].re * m, taus[q].im * m);
    if (p.i > 0) row[c - 1] = mk(-f.xl, 0.0);
    if (p.i < L.nx - 1) row[c + 1] = mk(-f.xh, 0.0);
    if (p.j > 0) row[c - L.nx] = mk(-f.yl, 0.0);
    if (p.j < L.ny - 1) row[c + L.nx] = mk(-f.yh, 0.0);
    if (L.nz > 1) {
      if (p.k > 0) row[c - sxy] = mk(-f.zl, 0.0);
      if (p.k < L.nz - 1) row[c + sxy] = mk(-f.zh, 0.0);
    }
  }
}

// --------------------------------------------------------------------- apply
// y = (K + s M) x; the shift is `s` or, with `st`, taus[st[slot].tau].
template <typename T>
__global__ void k_apply(LevelView<T> L, z64 s_fixed, const SlotState* st, const z64* taus,
                        const cx<T>* __restrict__ x, cx<T>* __restrict__ y, int64_t vs) {
  int slot = blockIdx.z;
  Cell p;
  int c;
  if (!grid_cell(L.nx, L.ny, L.nz, &p, &c)) return;
  z64 s = st ? taus[st[slot].tau] : s_fixed;
  y[slot * vs + c] = apply_at(L, p, c, cvt<T>(s), x + slot * vs);
}

// --------------------------------------------------------------------- smoother
// One red-black Gauss-Seidel half sweep on the cells of `color`
// (color 0 = red: i + j + k even): z_c = (f_c + sum_nb t z_nb) / (K_cc + tau M_cc).
// `zero_start`: the other colour is taken as zero (first sweep from z = 0).
// Multiple sources (SpMM form): a block holds G sources of the batch as
// threadIdx.z over the same cells (blockDim = (32, 8 / G, G)), so a cell's
// faces and inverse diagonal are fetched from memory once and served to the
// other sources' warps from the SM's L1 (sources in lockstep share tau_k);
// sources whose inner solve has finished return at once. Every source's update
// is the single-source one.
template <typename T, typename C>
__global__ void k_gs(LevelView<T, C> L, const SlotState* st, const cx<T>* __restrict__ invd,
                     const cx<T>* __restrict__ f, cx<T>* __restrict__ z, int64_t vs, int color, int zero_start,
                     int nslot) {
  pdl_enter();
  const int slot = blockIdx.z * blockDim.z + threadIdx.z;
  if (slot >= nslot || !slot_running(st, slot)) return;
  const int ii = blockIdx.x * GX + threadIdx.x;
  const int row = blockIdx.y * blockDim.y + threadIdx.y;
  if (row >= L.ny * L.nz) return;
  const int k = row / L.ny, j = row - k * L.ny;
  const int i = 2 * ii + ((j + k + color) & 1);
  if (i >= L.nx) return;
  const int c = row * L.nx + i;
  const cx<T> id = invd[(int64_t)st[slot].tau * L.n + c];
  z[slot * vs + c] = gs_value(L, Cell{i, j, k}, c, id, f + slot * vs, z + slot * vs, zero_start);
}

// The last half sweep of the finest level's post-smoothing fused with the
// defect correction: thread (ii, row) owns cells 2 ii and 2 ii + 1 of the row,
// updates the one of colour `color` as k_gs does, and adds both final values
// e to column k - 1 of the outer iterates (z_k = e on the first cycle, z_k + e
// after), the update of k_correct. z itself is not written: nothing reads the
// finest level's correction after this. Sources as in k_gs.
template <typename T, typename C>
__global__ void k_gs_correct(LevelView<T, C> L, const SlotState* st, const cx<T>* __restrict__ invd,
                             const cx<T>* __restrict__ f, const cx<T>* __restrict__ z, int64_t vs, int color,
                             z64* __restrict__ Zk, int64_t vsZk, int64_t zcol, int nslot) {
  pdl_enter();
  const int slot = blockIdx.z * blockDim.z + threadIdx.z;
  if (slot >= nslot || !slot_running(st, slot)) return;
  const int ii = blockIdx.x * GX + threadIdx.x;
  const int row = blockIdx.y * blockDim.y + threadIdx.y;
  if (row >= L.ny * L.nz || 2 * ii >= L.nx) return;
  const int k = row / L.ny, j = row - k * L.ny;
  const cx<T>* zs = z + slot * vs;
  z64* zk = Zk + slot * vsZk + (int64_t)(st[slot].k - 1) * zcol;
  const bool first = st[slot].cycles == 0;
  for (int h = 0; h < 2; ++h) {
    const int i = 2 * ii + h;
    if (i >= L.nx) break;
    const int c = row * L.nx + i;
    cx<T> e;
    if (((i + j + k) & 1) == color) {
      const cx<T> id = invd[(int64_t)st[slot].tau * L.n + c];
      e = gs_value(L, Cell{i, j, k}, c, id, f + slot * vs, zs, 0);
    } else {
      e = zs[c];
    }
    const z64 ev = cvt<double>(e);
    zk[c] = first ? ev : (zk[c] + ev);
  }
}

// --------------------------------------------------------------------- transfer
// Coarse right-hand side = sum over the children of the fine residual f - A z.
// Sources as in k_gs (threadIdx.z), so the children's coefficients come from
// memory once per block.
template <typename T, typename C>
__global__ void k_residual_restrict(LevelView<T, C> F, int rx, int ry, int rz, int cnx, int cny, int cnz,
                                    const SlotState* st, const z64* taus, const cx<T>* __restrict__ f,
                                    const cx<T>* __restrict__ z, int64_t vs, cx<T>* __restrict__ fc, int64_t vsc,
                                    int nslot) {
  pdl_enter();
  const int slot = blockIdx.z * blockDim.z + threadIdx.z;
  if (slot >= nslot || !slot_running(st, slot)) return;
  const int I = blockIdx.x * GX + threadIdx.x;
  const int row = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= cnx || row >= cny * cnz) return;
  const int K = row / cny, J = row - K * cny;
  const cx<T> s = cvt<T>(taus[st[slot].tau]);
  fc[slot * vsc + (int64_t)row * cnx + I] = restrict_value(F, rx, ry, rz, I, J, K, s, f + slot * vs, z + slot * vs);
}

// Coarse right-hand side on a 3D level coarsened by 2 in every axis, one
// source per block. The per-coarse-cell loop of k_residual_restrict computes
// its eight children one after another; here the block's 256 threads first
// compute the fine residuals f - A z of a 32 x 8 x 2 tile, one (i, j) column
// of two planes each, into shared memory, then one thread per coarse cell
// adds its children in restrict_value's order (z, then y, then x child),
// skipping those past the fine grid, so the sum is bitwise the same.
template <typename T, typename C>
__global__ void __launch_bounds__(256) k_residual_restrict3(LevelView<T, C> F, int cnx, int cny, int cnz,
                                                            const SlotState* st, const z64* taus,
                                                            const cx<T>* __restrict__ f, const cx<T>* __restrict__ z,
                                                            int64_t vs, cx<T>* __restrict__ fc, int64_t vsc) {
  pdl_enter();
  __shared__ cx<T> sr[2][GY][GX];
  const int slot = blockIdx.z;
  if (!slot_running(st, slot)) return;
  const int nby = (F.ny + GY - 1) / GY;
  const int K = blockIdx.y / nby, by = blockIdx.y - K * nby;
  const int i = blockIdx.x * GX + threadIdx.x, j = by * GY + threadIdx.y;
  const cx<T> s = cvt<T>(taus[st[slot].tau]);
  const cx<T>* fs = f + slot * vs;
  const cx<T>* zs = z + slot * vs;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int k = 2 * K + q;
    cx<T> r = mk(T(0), T(0));
    if (i < F.nx && j < F.ny && k < F.nz) {
      const int64_t cc = ((int64_t)k * F.ny + j) * F.nx + i;
      r = fs[cc] - apply_at(F, Cell{i, j, k}, cc, s, zs);
    }
    sr[q][threadIdx.y][threadIdx.x] = r;
  }
  __syncthreads();
  const int t = threadIdx.y * GX + threadIdx.x;
  if (t >= (GX / 2) * (GY / 2)) return;
  const int ti = t % (GX / 2), tj = t / (GX / 2);
  const int I = blockIdx.x * (GX / 2) + ti, J = by * (GY / 2) + tj;
  if (I >= cnx || J >= cny) return;
  cx<T> acc = mk(T(0), T(0));
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        if (2 * I + a >= F.nx || 2 * J + b >= F.ny || 2 * K + c >= F.nz) continue;
        acc = acc + sr[c][2 * tj + b][2 * ti + a];
      }
  fc[slot * vsc + ((int64_t)K * cny + J) * cnx + I] = acc;
}

// z_fine += P z_coarse
template <typename T>
__global__ void k_prolong_add(LevelView<T> F, int rx, int ry, int rz, int cnx, int cny, int cnz, uint32_t mask,
                              const SlotState* st, const cx<T>* __restrict__ zc, int64_t vsc,
                              cx<T>* __restrict__ z, int64_t vs) {
  pdl_enter();
  int slot = blockIdx.z;
  if (!slot_running(st, slot)) return;
  Cell p;
  int c;
  if (!grid_cell(F.nx, F.ny, F.nz, &p, &c)) return;
  cx<T>* zs = z + slot * vs;
  zs[c] = zs[c] + prolong_value(p, rx, ry, rz, cnx, cny, cnz, mask, zc + slot * vsc);
}

// z_fine += P z_coarse on a 3D level coarsened by 2 in every axis: a block
// updates 32 x 8 cells in each of the two fine planes of coarse plane K and
// first stages the 18 x 6 x 3 coarse values they interpolate from (planes K -
// 1, K and K + 1) in shared memory, so each coarse value is read once per
// block instead of once per fine cell; the interpolation itself is
// prolong_value_at's, on those values.
template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add3(LevelView<T> F, int cnx, int cny, int cnz, uint32_t mask,
                                                      const SlotState* st, const cx<T>* __restrict__ zc,
                                                      int64_t vsc, cx<T>* __restrict__ z, int64_t vs) {
  pdl_enter();
  constexpr int SX = GX / 2 + 2, SY = GY / 2 + 2;
  __shared__ cx<T> sc[3][SY][SX];
  const int slot = blockIdx.z;
  if (!slot_running(st, slot)) return;
  const int nby = (F.ny + GY - 1) / GY;
  const int K = blockIdx.y / nby, by = blockIdx.y - K * nby;
  const int x0 = blockIdx.x * GX, y0 = by * GY;
  const int X0 = x0 / 2 - 1, Y0 = y0 / 2 - 1;
  const cx<T>* zcs = zc + slot * vsc;
  // the cells' own values are loaded before the staging barrier, so their
  // latency overlaps that of the coarse values
  const int i = x0 + threadIdx.x, j = y0 + threadIdx.y;
  cx<T>* zs = z + slot * vs;
  bool own[2];
  int64_t c[2];
  cx<T> z0[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int k = 2 * K + q;
    own[q] = i < F.nx && j < F.ny && k < F.nz;
    c[q] = ((int64_t)k * F.ny + j) * F.nx + i;
    z0[q] = own[q] ? zs[c[q]] : mk(T(0), T(0));
  }
  for (int t = threadIdx.y * GX + threadIdx.x; t < 3 * SY * SX; t += GX * GY) {
    const int q = t / (SY * SX), rem = t - q * (SY * SX);
    const int yy = rem / SX, xx = rem - yy * SX;
    const int X = X0 + xx, Y = Y0 + yy, Z = K - 1 + q;
    const bool in = X >= 0 && X < cnx && Y >= 0 && Y < cny && Z >= 0 && Z < cnz;
    sc[q][yy][xx] = in ? zcs[((int64_t)Z * cny + Y) * cnx + X] : mk(T(0), T(0));
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (!own[q]) continue;
    zs[c[q]] = z0[q] + prolong_value_at<T>(Cell{i, j, 2 * K + q}, 2, 2, 2, cnx, cny, cnz, mask,
                                            [&](int X, int Y, int Z) { return sc[Z - K + 1][Y - Y0][X - X0]; });
  }
}

// --------------------------------------------------------------------- fused 2D level kernels
// One level of the V-cycle on a 2D grid coarsened in both axes, in two
// kernels over TX x TY tiles with a halo of H = 4 cells held in shared memory.
// Red-black half sweeps only read the other colour, so every half sweep is
// recomputed on a region that shrinks by one cell per sweep; the tile interior
// then holds exactly the values of the per-sweep kernels.
//   pre : z = four half sweeps from z = 0 (red, black, red, black); write z;
//         coarse f = sum over children of (f - A z)
//   post: z += P z_coarse; four half sweeps (black, red, black, red); write z
constexpr int DEFECT_ROWS = 2;  // rows of cells per thread in the defect kernel

// sum over existing neighbours of t_face * z_nb for a 2D cell held at r in a
// shared tile of row length RX (same order as nb_sum)
template <typename T>
__device__ __forceinline__ cx<T> nb_sum_tile(const LevelView<T>& L, Cell p, int r, int RX, const cx<T>* sZ,
                                             cx<T> s0 = cx<T>{T(0), T(0)}) {
  Faces<T> f = faces_at(L, p);
  cx<T> s = s0;
  if (p.i > 0) s = axpy(f.xl, sZ[r - 1], s);
  if (p.i < L.nx - 1) s = axpy(f.xh, sZ[r + 1], s);
  if (p.j > 0) s = axpy(f.yl, sZ[r - RX], s);
  if (p.j < L.ny - 1) s = axpy(f.yh, sZ[r + RX], s);
  return s;
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (TX == 32 ? 6 : 8) : 4) k_pre2d(LevelView<T> L, const SlotState* st, const cx<T>* __restrict__ invd,
                                               const z64* taus, const cx<T>* __restrict__ f, cx<T>* __restrict__ z,
                                               int64_t vs, cx<T>* __restrict__ fc, int64_t vsc) {
  pdl_enter();
  constexpr int RX = TX + 2 * FH, RY = TY + 2 * FH;
  extern __shared__ __align__(16) unsigned char pre_smem[];
  cx<T>* sF = (cx<T>*)pre_smem;
  cx<T>* sZ = sF + RX * RY;
  int slot = blockIdx.z;
  if (!slot_running(st, slot)) return;
  const int tau = st[slot].tau;
  const cx<T> sft = cvt<T>(taus[tau]);
  const cx<T>* ID = invd + (int64_t)tau * L.n;
  const cx<T>* fs = f + slot * vs;
  const int x0 = blockIdx.x * TX - FH, y0 = blockIdx.y * TY - FH;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int q = tid; q < RX * RY; q += nt) {
    int ry = q / RX, rx = q - ry * RX;
    int gx = x0 + rx, gy = y0 + ry;
    bool in = gx >= 0 && gx < L.nx && gy >= 0 && gy < L.ny;
    sF[q] = in ? fs[gy * L.nx + gx] : mk(T(0), T(0));
  }
  __syncthreads();
  for (int hs = 0; hs < 4; ++hs) {
    const int color = hs & 1;
    const int w = RX - 2 * hs, hgt = RY - 2 * hs;
    const int wh = (w + 1) >> 1;
    for (int q = tid; q < wh * hgt; q += nt) {
      int yy = q / wh;
      int ry = hs + yy;
      int gy = y0 + ry;
      int rx0 = hs + 2 * (q - yy * wh);
      int gx = x0 + rx0;
      if (((gx + gy) & 1) != color) { ++gx; ++rx0; }
      if (rx0 >= RX - hs || gx < 0 || gx >= L.nx || gy < 0 || gy >= L.ny) continue;
      int r = ry * RX + rx0;
      int c = gy * L.nx + gx;
      cx<T> rhs = sF[r];
      if (hs > 0) rhs = nb_sum_tile(L, Cell{gx, gy, 0}, r, RX, sZ, rhs);
      sZ[r] = ID[c] * rhs;
    }
    __syncthreads();
  }
  cx<T>* zs = z + slot * vs;
  for (int q = tid; q < TX * TY; q += nt) {
    int yy = q / TX, xx = q - yy * TX;
    int gx = x0 + FH + xx, gy = y0 + FH + yy;
    if (gx < L.nx && gy < L.ny) zs[gy * L.nx + gx] = sZ[(yy + FH) * RX + xx + FH];
  }
  // residual + restriction to the (TX/2) x (TY/2) coarse cells of the tile
  const int cnx = L.nx >> 1, cny = L.ny >> 1;
  cx<T>* fcs = fc + slot * vsc;
  for (int q = tid; q < (TX / 2) * (TY / 2); q += nt) {
    int Yl = q / (TX / 2), Xl = q - Yl * (TX / 2);
    int X = blockIdx.x * (TX / 2) + Xl, Y = blockIdx.y * (TY / 2) + Yl;
    if (X >= cnx || Y >= cny) continue;
    cx<T> acc = mk(T(0), T(0));
#pragma unroll 1
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        int gx = 2 * X + a, gy = 2 * Y + b;
        int r = (gy - y0) * RX + (gx - x0);
        int c = gy * L.nx + gx;
        Faces<T> fa = faces_at(L, Cell{gx, gy, 0});
        T d = fsum(fa), m = L.mm[c];
        cx<T> Az = mk(fmaT(sft.re, m, d), mulT(sft.im, m)) * sZ[r] - nb_sum_tile(L, Cell{gx, gy, 0}, r, RX, sZ);
        acc = acc + (sF[r] - Az);
      }
    fcs[Y * cnx + X] = acc;
  }
}

// post reads the pre-smoothed z and writes zout (a different buffer): tiles
// read their neighbours' cells as halo, which those tiles overwrite. With Zk
// given (finest level), the result e is instead added to the outer iterate,
// z_k = e on the first cycle and z_k + e after (the update of k_correct).
template <typename T, int TX, int TY>
__global__ void __launch_bounds__(256) k_post2d(LevelView<T> L, uint32_t mask, const SlotState* st,
                                                const cx<T>* __restrict__ invd, const cx<T>* __restrict__ f,
                                                const cx<T>* __restrict__ z, cx<T>* __restrict__ zout, int64_t vs,
                                                const cx<T>* __restrict__ zc, int64_t vsc, z64* __restrict__ Zk,
                                                int64_t vsZk, int64_t zcol) {
  pdl_enter();
  constexpr int RX = TX + 2 * FH, RY = TY + 2 * FH;
  extern __shared__ __align__(16) unsigned char post_smem[];
  cx<T>* sF = (cx<T>*)post_smem;
  cx<T>* sZ = sF + RX * RY;
  int slot = blockIdx.z;
  if (!slot_running(st, slot)) return;
  const int tau = st[slot].tau;
  const cx<T>* ID = invd + (int64_t)tau * L.n;
  const cx<T>* fs = f + slot * vs;
  const cx<T>* zs = z + slot * vs;
  cx<T>* zo = zout + slot * vs;
  const cx<T>* zcs = zc + slot * vsc;
  const int cnx = L.nx >> 1, cny = L.ny >> 1;
  const int x0 = blockIdx.x * TX - FH, y0 = blockIdx.y * TY - FH;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int q = tid; q < RX * RY; q += nt) {
    int ry = q / RX, rx = q - ry * RX;
    int gx = x0 + rx, gy = y0 + ry;
    bool in = gx >= 0 && gx < L.nx && gy >= 0 && gy < L.ny;
    if (in) {
      int c = gy * L.nx + gx;
      sF[q] = fs[c];
      sZ[q] = zs[c] + prolong_value(Cell{gx, gy, 0}, 2, 2, 1, cnx, cny, 1, mask, zcs);
    } else {
      sF[q] = mk(T(0), T(0));
      sZ[q] = mk(T(0), T(0));
    }
  }
  __syncthreads();
  for (int hs = 0; hs < 4; ++hs) {
    const int color = (hs & 1) ? 0 : 1;  // black, red, black, red
    const int sh = hs + 1;
    const int w = RX - 2 * sh, hgt = RY - 2 * sh;
    const int wh = (w + 1) >> 1;
    for (int q = tid; q < wh * hgt; q += nt) {
      int yy = q / wh;
      int ry = sh + yy;
      int gy = y0 + ry;
      int rx0 = sh + 2 * (q - yy * wh);
      int gx = x0 + rx0;
      if (((gx + gy) & 1) != color) { ++gx; ++rx0; }
      if (rx0 >= RX - sh || gx < 0 || gx >= L.nx || gy < 0 || gy >= L.ny) continue;
      int r = ry * RX + rx0;
      int c = gy * L.nx + gx;
      cx<T> rhs = nb_sum_tile(L, Cell{gx, gy, 0}, r, RX, sZ, sF[r]);
      sZ[r] = ID[c] * rhs;
    }
    __syncthreads();
  }
  if (Zk) {
    z64* zk = Zk + slot * vsZk + (int64_t)(st[slot].k - 1) * zcol;
    const bool first = st[slot].cycles == 0;
    for (int q = tid; q < TX * TY; q += nt) {
      int yy = q / TX, xx = q - yy * TX;
      int gx = x0 + FH + xx, gy = y0 + FH + yy;
      if (gx < L.nx && gy < L.ny) {
        const int c = gy * L.nx + gx;
        const z64 ev = cvt<double>(sZ[(yy + FH) * RX + xx + FH]);
        zk[c] = first ? ev : (zk[c] + ev);
      }
    }
    return;
  }
  for (int q = tid; q < TX * TY; q += nt) {
    int yy = q / TX, xx = q - yy * TX;
    int gx = x0 + FH + xx, gy = y0 + FH + yy;
    if (gx < L.nx && gy < L.ny) zo[gy * L.nx + gx] = sZ[(yy + FH) * RX + xx + FH];
  }
}

// --------------------------------------------------------------------- tail
// The V-cycle of every level from `lt` down (levels small enough for one CTA)
// in one kernel: one block per slot, level vectors in shared memory,
// coefficients read through the cache. Same operations, in the same order, as
// the per-level kernels.
template <typename T>
__global__ void __launch_bounds__(TAIL_THREADS, 1) k_tail_vcycle(TailParams<T> P, const SlotState* st) {
  pdl_enter();
  int slot = blockIdx.x;
  if (!slot_running(st, slot)) return;
  extern __shared__ __align__(16) unsigned char tail_smem[];
  __shared__ LevelView<T> SV[MAX_LEVELS];
  __shared__ const cx<T>* SI[MAX_LEVELS];
  cx<T>* sh = (cx<T>*)tail_smem;
  const int tau = st[slot].tau;
  const cx<T> sft = cvt<T>(P.taus[tau]);
  const int nt = blockDim.x, tid = threadIdx.x;
  // level views: coefficients staged in shared memory (one bulk copy) or read from global
  if (tid < P.nlev) {
    const TailLevel<T>& A = P.lev[tid];
    LevelView<T> v = A.L;
    const cx<T>* id = A.invd + (int64_t)tau * A.L.n;
    if (P.staged) {
      int nfx = (v.nx + 1) * v.ny * v.nz, nfy = v.nx * (v.ny + 1) * v.nz;
      int nfz = v.nz > 1 ? v.nx * v.ny * (v.nz + 1) : 0;
      T* base = (T*)(tail_smem + A.cbyte);
      v.fx = base;
      v.fy = base + nfx;
      v.fz = base + nfx + nfy;
      v.mm = base + nfx + nfy + nfz;
      int realn = nfx + nfy + nfz + v.n;
      realn = (realn + 3) & ~3;
      id = (const cx<T>*)(base + realn);
    }
    SV[tid] = v;
    SI[tid] = id;
  }
  if (P.staged && P.blob) {
    // one flat copy of this tau's coefficients of all tail levels
    const uint4* src = (const uint4*)(P.blob + (size_t)tau * P.blob_bytes);
    uint4* dst = (uint4*)(tail_smem + P.coef0);
    for (int q = tid; q < P.blob_bytes / 16; q += nt) dst[q] = src[q];
  }
  __syncthreads();
  if (P.staged && !P.blob) {
    for (int l = 0; l < P.nlev; ++l) {
      const TailLevel<T>& A = P.lev[l];
      const LevelView<T>& v = SV[l];
      int nfx = (v.nx + 1) * v.ny * v.nz, nfy = v.nx * (v.ny + 1) * v.nz;
      int nfz = v.nz > 1 ? v.nx * v.ny * (v.nz + 1) : 0;
      T* dfx = (T*)v.fx;
      for (int q = tid; q < nfx; q += nt) dfx[q] = A.L.fx[q];
      T* dfy = (T*)v.fy;
      for (int q = tid; q < nfy; q += nt) dfy[q] = A.L.fy[q];
      T* dfz = (T*)v.fz;
      for (int q = tid; q < nfz; q += nt) dfz[q] = A.L.fz[q];
      T* dmm = (T*)v.mm;
      for (int q = tid; q < v.n; q += nt) dmm[q] = A.L.mm[q];
      cx<T>* did = (cx<T>*)SI[l];
      const cx<T>* gid = A.invd + (int64_t)tau * v.n;
      for (int q = tid; q < v.n; q += nt) did[q] = gid[q];
    }
  }
  {
    const TailLevel<T>& A = P.lev[0];
    const cx<T>* fin = P.f_in + slot * P.vs;
    for (int c = tid; c < A.L.n; c += nt) sh[A.off + c] = fin[c];
  }
  __syncthreads();
  auto sweep = [&](int l, int color, int zs) {
    const LevelView<T> L = SV[l];  // a register copy: the loop's shared-memory stores cannot alias it
    cx<T>* F = sh + P.lev[l].off;
    cx<T>* Z = F + L.n;
    const cx<T>* ID = SI[l];
    int work = ((L.nx + 1) >> 1) * L.ny * L.nz;
    for (int t = tid; t < work; t += nt) {
      Cell p;
      int c;
      if (color_cell(L.nx, L.ny, L.nz, color, t, &p, &c)) Z[c] = gs_value(L, p, c, ID[c], F, Z, zs);
    }
    __syncthreads();
  };
  for (int l = 0; l + 1 < P.nlev; ++l) {
    const TailLevel<T>& A = P.lev[l];
    const TailLevel<T>& B = P.lev[l + 1];
    for (int r = 0; r < 2; ++r) {
      sweep(l, 0, r == 0);
      sweep(l, 1, 0);
    }
    cx<T>* F = sh + A.off;
    cx<T>* Z = F + A.L.n;
    cx<T>* FC = sh + B.off;
    const LevelView<T> LA = SV[l];
    for (int C = tid; C < B.L.n; C += nt) {
      Cell pc = cell_of(C, B.L.nx, B.L.ny);
      FC[C] = restrict_value(LA, A.rx, A.ry, A.rz, pc.i, pc.j, pc.k, sft, F, Z);
    }
    __syncthreads();
  }
  {
    const TailLevel<T>& Cl = P.lev[P.nlev - 1];
    const cx<T>* F = sh + Cl.off;
    cx<T>* Z = sh + Cl.off + Cl.L.n;
    const cx<T>* Ainv = P.Ainv + (int64_t)tau * P.nc * P.nc;
    for (int r = tid; r < P.nc; r += nt) {
      cx<T> acc = mk(T(0), T(0));
      const cx<T>* row = Ainv + (int64_t)r * P.nc;
      for (int l = 0; l < P.nc; ++l) acc = acc + row[l] * F[l];
      Z[r] = acc;
    }
    __syncthreads();
  }
  for (int l = P.nlev - 2; l >= 0; --l) {
    const TailLevel<T>& A = P.lev[l];
    const TailLevel<T>& B = P.lev[l + 1];
    cx<T>* Z = sh + A.off + A.L.n;
    const cx<T>* ZC = sh + B.off + B.L.n;
    for (int c = tid; c < A.L.n; c += nt) {
      Cell p = cell_of(c, A.L.nx, A.L.ny);
      Z[c] = Z[c] + prolong_value(p, A.rx, A.ry, A.rz, B.L.nx, B.L.ny, B.L.nz, P.mask, ZC);
    }
    __syncthreads();
    for (int r = 0; r < 2; ++r) {
      sweep(l, 1, 0);
      sweep(l, 0, 0);
    }
  }
  {
    const TailLevel<T>& A = P.lev[0];
    cx<T>* zout = P.z_out + slot * P.vs;
    const cx<T>* Z = sh + A.off + A.L.n;
    for (int c = tid; c < A.L.n; c += nt) zout[c] = Z[c];
  }
}

// --------------------------------------------------------------------- 2D tail
// The tail V-cycle for 2D levels halved in both axes, with the cells of every
// level owned in horizontal pairs: thread t owns cells 2t and 2t + 1 of the
// level it is on (one red, one black, as nx is even), and keeps their faces,
// storage, inverse diagonals, right-hand sides and iterates in registers for
// the whole visit of the level; only the iterates go through shared memory,
// for the neighbours. Each cell update performs the operations of gs_value,
// restrict_value and prolong_value in the same order as k_tail_vcycle.
template <typename T>
struct TailPair {
  int i0, j, c0;
  bool own;
  T fxa, fxb, fxc;           // x faces left of c0, between, right of c1
  T yl0, yh0, yl1, yh1;      // y faces of c0 and c1
  T m0, m1;
  cx<T> id0, id1, f0, f1, z0, z1;
};

template <typename T>
__device__ __forceinline__ void tail2d_load(const TailLevel<T>& A, const unsigned char* smem, const cx<T>* F, int t,
                                            int tau, TailPair<T>& q) {
  const int nx = A.L.nx, ny = A.L.ny;
  const int n = nx * ny;
  q.own = 2 * t < n;
  if (!q.own) return;
  q.c0 = 2 * t;
  q.j = q.c0 / nx;
  q.i0 = q.c0 - q.j * nx;
  const int nfx = (nx + 1) * ny, nfy = nx * (ny + 1);
  const T* fx = (const T*)(smem + A.cbyte);
  const T* fy = fx + nfx;
  const T* mm = fy + nfy;
  const cx<T>* id = (const cx<T>*)(fx + ((nfx + nfy + n + 3) & ~3));
  const int rx = q.j * (nx + 1) + q.i0;
  q.fxa = fx[rx];
  q.fxb = fx[rx + 1];
  q.fxc = fx[rx + 2];
  q.yl0 = fy[q.c0];
  q.yl1 = fy[q.c0 + 1];
  q.yh0 = fy[q.c0 + nx];
  q.yh1 = fy[q.c0 + nx + 1];
  q.m0 = mm[q.c0];
  q.m1 = mm[q.c0 + 1];
  q.id0 = id[q.c0];
  q.id1 = id[q.c0 + 1];
  q.f0 = F[q.c0];
  q.f1 = F[q.c0 + 1];
  (void)tau;
}

// half sweep of `color` on the owned cell of that colour
template <typename T>
__device__ __forceinline__ void tail2d_gs(TailPair<T>& q, int nx, int ny, cx<T>* Z, int color, int zs) {
  if (!q.own) return;
  const bool first = ((q.j & 1) == color);  // c0 = (i0 even, j) has colour j & 1
  if (first) {
    cx<T> rhs = q.f0;
    if (!zs) {
      if (q.i0 > 0) rhs = axpy(q.fxa, Z[q.c0 - 1], rhs);
      rhs = axpy(q.fxb, q.z1, rhs);
      if (q.j > 0) rhs = axpy(q.yl0, Z[q.c0 - nx], rhs);
      if (q.j < ny - 1) rhs = axpy(q.yh0, Z[q.c0 + nx], rhs);
    }
    q.z0 = q.id0 * rhs;
    Z[q.c0] = q.z0;
  } else {
    cx<T> rhs = q.f1;
    if (!zs) {
      rhs = axpy(q.fxb, q.z0, rhs);
      if (q.i0 + 1 < nx - 1) rhs = axpy(q.fxc, Z[q.c0 + 2], rhs);
      if (q.j > 0) rhs = axpy(q.yl1, Z[q.c0 + 1 - nx], rhs);
      if (q.j < ny - 1) rhs = axpy(q.yh1, Z[q.c0 + 1 + nx], rhs);
    }
    q.z1 = q.id1 * rhs;
    Z[q.c0 + 1] = q.z1;
  }
}

// f - (K + s M) z on the two owned cells (apply_at with d the sum of the faces)
template <typename T>
__device__ __forceinline__ void tail2d_residual(const TailPair<T>& q, int nx, int ny, const cx<T>* Z, cx<T> s,
                                                cx<T>* r0, cx<T>* r1) {
  const T zero = T(0);
  {
    Faces<T> fa{q.fxa, q.fxb, q.yl0, q.yh0, zero, zero};
    const T d = fsum(fa);
    cx<T> nb = mk(zero, zero);
    if (q.i0 > 0) nb = axpy(q.fxa, Z[q.c0 - 1], nb);
    nb = axpy(q.fxb, q.z1, nb);
    if (q.j > 0) nb = axpy(q.yl0, Z[q.c0 - nx], nb);
    if (q.j < ny - 1) nb = axpy(q.yh0, Z[q.c0 + nx], nb);
    *r0 = q.f0 - (mk(fmaT(s.re, q.m0, d), mulT(s.im, q.m0)) * q.z0 - nb);
  }
  {
    Faces<T> fa{q.fxb, q.fxc, q.yl1, q.yh1, zero, zero};
    const T d = fsum(fa);
    cx<T> nb = mk(zero, zero);
    nb = axpy(q.fxb, q.z0, nb);
    if (q.i0 + 1 < nx - 1) nb = axpy(q.fxc, Z[q.c0 + 2], nb);
    if (q.j > 0) nb = axpy(q.yl1, Z[q.c0 + 1 - nx], nb);
    if (q.j < ny - 1) nb = axpy(q.yh1, Z[q.c0 + 1 + nx], nb);
    *r1 = q.f1 - (mk(fmaT(s.re, q.m1, d), mulT(s.im, q.m1)) * q.z1 - nb);
  }
}

template <typename T>
__global__ void __launch_bounds__(TAIL_THREADS, 1) k_tail2d(TailParams<T> P, const SlotState* st) {
  pdl_enter();
  const int slot = blockIdx.x;
  if (!slot_running(st, slot)) return;
  extern __shared__ __align__(16) unsigned char t2_smem[];
  cx<T>* sh = (cx<T>*)t2_smem;
  const int tau = st[slot].tau;
  const cx<T> sft = cvt<T>(P.taus[tau]);
  const int nt = blockDim.x, tid = threadIdx.x;
  {
    const uint4* src = (const uint4*)(P.blob + (size_t)tau * P.blob_bytes);
    uint4* dst = (uint4*)(t2_smem + P.coef0);
    for (int q = tid; q < P.blob_bytes / 16; q += nt) dst[q] = src[q];
    const cx<T>* ag = P.Ainv + (int64_t)tau * P.nc * P.nc;
    cx<T>* as = (cx<T>*)(t2_smem + P.ainv_off);
    for (int q = tid; q < P.nc * P.nc; q += nt) as[q] = ag[q];
    const TailLevel<T>& A = P.lev[0];
    const cx<T>* fin = P.f_in + slot * P.vs;
    for (int c = tid; c < A.L.n; c += nt) sh[A.off + c] = fin[c];
  }
  __syncthreads();
  TailPair<T> q;
  // ---- down
  for (int l = 0; l + 1 < P.nlev; ++l) {
    const TailLevel<T>& A = P.lev[l];
    const TailLevel<T>& B = P.lev[l + 1];
    const int nx = A.L.nx, ny = A.L.ny;
    cx<T>* F = sh + A.off;
    cx<T>* Z = F + A.L.n;
    tail2d_load(A, t2_smem, F, tid, tau, q);
    for (int r = 0; r < 2; ++r) {
      tail2d_gs(q, nx, ny, Z, 0, r == 0);
      __syncthreads();
      tail2d_gs(q, nx, ny, Z, 1, 0);
      __syncthreads();
    }
    // restriction: the pair in row 2J sums its two residuals, the pair in
    // row 2J + 1 adds its own onto that (the child order of restrict_value)
    const int cnx = B.L.nx;
    cx<T>* FC = sh + B.off;
    cx<T>* S = FC + B.L.n;  // the coarse iterate's storage, free until its first sweep
    cx<T> r0, r1;
    if (q.own) {
      tail2d_residual(q, nx, ny, Z, sft, &r0, &r1);
      if ((q.j & 1) == 0) S[(q.j >> 1) * cnx + (q.i0 >> 1)] = (mk(T(0), T(0)) + r0) + r1;
    }
    __syncthreads();
    if (q.own && (q.j & 1)) {
      const int C = (q.j >> 1) * cnx + (q.i0 >> 1);
      FC[C] = (S[C] + r0) + r1;
    }
    __syncthreads();
  }
  {
    const TailLevel<T>& Cl = P.lev[P.nlev - 1];
    const cx<T>* F = sh + Cl.off;
    cx<T>* Z = sh + Cl.off + Cl.L.n;
    const cx<T>* Ainv = (const cx<T>*)(t2_smem + P.ainv_off);
    for (int r = tid; r < P.nc; r += nt) {
      cx<T> acc = mk(T(0), T(0));
      const cx<T>* row = Ainv + r * P.nc;
      for (int l = 0; l < P.nc; ++l) acc = acc + row[l] * F[l];
      Z[r] = acc;
    }
    __syncthreads();
  }
  if (P.nlev == 1) {
    const TailLevel<T>& A = P.lev[0];
    cx<T>* zout = P.z_out + slot * P.vs;
    const cx<T>* Z = sh + A.off + A.L.n;
    for (int c = tid; c < A.L.n; c += nt) zout[c] = Z[c];
    return;
  }
  // ---- up
  for (int l = P.nlev - 2; l >= 0; --l) {
    const TailLevel<T>& A = P.lev[l];
    const TailLevel<T>& B = P.lev[l + 1];
    const int nx = A.L.nx, ny = A.L.ny;
    cx<T>* F = sh + A.off;
    cx<T>* Z = F + A.L.n;
    const cx<T>* ZC = sh + B.off + B.L.n;
    const int cnx = B.L.nx, cny = B.L.ny;
    tail2d_load(A, t2_smem, F, tid, tau, q);
    if (q.own) {
      auto get = [&](int X, int Y, int) { return ZC[Y * cnx + X]; };
      q.z0 = Z[q.c0] + prolong_value_at<T>(Cell{q.i0, q.j, 0}, 2, 2, 1, cnx, cny, 1, P.mask, get);
      q.z1 = Z[q.c0 + 1] + prolong_value_at<T>(Cell{q.i0 + 1, q.j, 0}, 2, 2, 1, cnx, cny, 1, P.mask, get);
      Z[q.c0] = q.z0;
      Z[q.c0 + 1] = q.z1;
    }
    __syncthreads();
    for (int r = 0; r < 2; ++r) {
      tail2d_gs(q, nx, ny, Z, 1, 0);
      __syncthreads();
      tail2d_gs(q, nx, ny, Z, 0, 0);
      __syncthreads();
    }
  }
  if (q.own) {
    cx<T>* zout = P.z_out + slot * P.vs;
    zout[q.c0] = q.z0;
    zout[q.c0 + 1] = q.z1;
  }
}

bool tail2d_ok(const std::vector<LevelHost>& Ls, int lt) {
  const int nl = (int)Ls.size();
  if (Ls[nl - 1].nz != 1) return false;
  for (int l = lt; l + 1 < nl; ++l) {
    const LevelHost& A = Ls[l];
    if (A.nz != 1 || A.rx != 2 || A.ry != 2 || A.nx % 2 || A.ny % 2 || A.n > 2 * TAIL_THREADS) return false;
  }
  return true;
}

// --------------------------------------------------------------------- coarsest
// Gauss-Jordan inversion with partial pivoting of one n x n complex matrix per
// block (blockIdx.x = tau index), in place on A (row-major) with the inverse
// written to Ainv. n <= MAX_COARSE.
__global__ void k_gauss_jordan(z64* A, z64* Ainv, int n, int* singular) {
  z64* a = A + (int64_t)blockIdx.x * n * n;
  z64* inv = Ainv + (int64_t)blockIdx.x * n * n;
  __shared__ int piv;
  __shared__ double best[1024];
  __shared__ int besti[1024];
  for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x)
    inv[t] = (t / n == t % n) ? mk(1.0, 0.0) : mk(0.0, 0.0);
  __syncthreads();
  for (int col = 0; col < n; ++col) {
    double bv = -1.0;
    int bi = col;
    for (int r = col + threadIdx.x; r < n; r += blockDim.x) {
      double v = abs2(a[(int64_t)r * n + col]);
      if (v > bv) { bv = v; bi = r; }
    }
    best[threadIdx.x] = bv;
    besti[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        double o = best[threadIdx.x + s];
        int oi = besti[threadIdx.x + s];
        if (o > best[threadIdx.x] || (o == best[threadIdx.x] && oi < besti[threadIdx.x])) {
          best[threadIdx.x] = o;
          besti[threadIdx.x] = oi;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      piv = besti[0];
      if (!(best[0] > 0.0)) *singular = 1;
    }
    __syncthreads();
    int pr = piv;
    if (pr != col) {
      for (int l = threadIdx.x; l < n; l += blockDim.x) {
        z64 t1 = a[(int64_t)pr * n + l];
        a[(int64_t)pr * n + l] = a[(int64_t)col * n + l];
        a[(int64_t)col * n + l] = t1;
        z64 t2 = inv[(int64_t)pr * n + l];
        inv[(int64_t)pr * n + l] = inv[(int64_t)col * n + l];
        inv[(int64_t)col * n + l] = t2;
      }
    }
    __syncthreads();
    z64 d = a[(int64_t)col * n + col];
    double den = abs2(d);
    z64 rd = den > 0.0 ? mk(d.re / den, -d.im / den) : mk(0.0, 0.0);
    __syncthreads();
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
      a[(int64_t)col * n + l] = rd * a[(int64_t)col * n + l];
      inv[(int64_t)col * n + l] = rd * inv[(int64_t)col * n + l];
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) {
      int r = (int)(t / n), l = (int)(t % n);
      if (r == col) continue;
      z64 fct = a[(int64_t)r * n + col];
      if (l != col) {
        a[t] = a[t] - fct * a[(int64_t)col * n + l];
      }
      inv[t] = inv[t] - fct * inv[(int64_t)col * n + l];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x)
      if (r != col) a[(int64_t)r * n + col] = mk(0.0, 0.0);
    __syncthreads();
  }
}

template <typename T>
__global__ void k_to_prec(const z64* __restrict__ a, cx<T>* __restrict__ b, int64_t n) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) b[t] = cvt<T>(a[t]);
}

// z = Ainv[tau] f on the coarsest level, one row per thread.
template <typename T>
__global__ void k_coarse_solve(const cx<T>* __restrict__ Ainv, int n, const SlotState* st,
                               const cx<T>* __restrict__ f, cx<T>* __restrict__ z, int64_t vs) {
  int slot = blockIdx.y;
  if (!slot_running(st, slot)) return;
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const cx<T>* a = Ainv + ((int64_t)st[slot].tau * n + r) * n;
  const cx<T>* fs = f + slot * vs;
  cx<T> acc = mk(T(0), T(0));
  for (int l = 0; l < n; ++l) acc = acc + a[l] * fs[l];
  z[slot * vs + r] = acc;
}

// --------------------------------------------------------------------- defect correction
// z += e (first cycle: z = e), z in fp64, e in the cycle precision.
template <typename T>
__global__ void k_correct(const SlotState* st, cx<double>* __restrict__ z, int64_t zs, int64_t zcol,
                          const cx<T>* __restrict__ e, int64_t es, int64_t n) {
  int slot = blockIdx.y;
  if (!slot_running(st, slot)) return;
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n) return;
  z64 ev = cvt<double>(e[slot * es + c]);
  z64* zp = z + slot * zs + (int64_t)(st[slot].k - 1) * zcol + c;
  *zp = st[slot].cycles == 0 ? ev : (*zp + ev);
}

// After the per-slot decisions: with `use_cond`, the last slot to report sets
// the graph's loop condition to "some slot still runs its inner solve"
// (flags[slot] collects the answers, counter[0] counts reports and is reset by
// the last one).
__device__ __forceinline__ void report_slot(int slot, int running, int nslot, int* flags, int* counter,
                                            cudaGraphConditionalHandle cond) {
  flags[slot] = running;
  __threadfence();
  if (atomicAdd(counter, 1) == nslot - 1) {
    __threadfence();
    int any = 0;
    for (int q = 0; q < nslot; ++q) any |= ((volatile int*)flags)[q];
    *counter = 0;
    cudaGraphSetConditional(cond, any ? 1u : 0u);
  }
}

// The inner-solve decision of one slot from ||p||^2 = a and ||v||^2 = b
// (Section 4: stop when ||p_k|| <= eps ||v_k||, or after max_cycles, or after the
// replayed number of cycles). Returns whether the slot keeps cycling.
__device__ __forceinline__ int decide_slot(SlotState& s, int slot, double a, double b, int first, double eps,
                                           int max_cycles, const int32_t* replay_cycles, int m_max, double relax,
                                           double tol) {
  eps = inner_eps(eps, relax, tol, s.rmax);
  s.pnorm2 = a;
  if (first) {
    s.vnorm2 = b;
    s.cycles = 0;
  } else {
    s.cycles += 1;
  }
  bool done;
  if (replay_cycles) done = s.cycles >= replay_cycles[(int64_t)slot * m_max + (s.k - 1)];
  else if (first) done = false;
  else {
    done = a <= eps * eps * s.vnorm2 || s.cycles >= max_cycles;
    if (!(a <= eps * eps * s.vnorm2) && s.cycles >= max_cycles) s.inner_capped = 1;
  }
  s.inner_done = done ? 1 : 0;
  return done ? 0 : 1;
}

struct DecideArgs {
  int on;                        // decide in the last block of each slot
  double eps;
  int max_cycles;
  const int32_t* replay_cycles;  // null unless replaying
  int m_max;
  int use_cond;
  cudaGraphConditionalHandle cond;
  int* flags;
  int* counter;
  int* bcount;                   // per-slot count of finished blocks, reset by the last one
  int nslot;
  double relax, tol;             // relaxed inner tolerance (relax <= 0: eps)
};

// r = v - (K + tau M) z in fp64; f0 = r in the cycle precision; per-block
// partial sums of |r|^2 (and |v|^2 when `with_v`). With D.on the last block of
// each slot sums the partials in a fixed order and takes the inner-solve
// decision (the work of k_inner_decide, without a launch of its own).
template <typename T>
__global__ void k_defect(LevelView<double> L, SlotState* st, const z64* taus, const z64* __restrict__ diag64,
                         const z64* __restrict__ v, int64_t vsv, const z64* __restrict__ z, int64_t vsz, int64_t col,
                         int zero_z, cx<T>* __restrict__ f0, int64_t vsf, double* __restrict__ partial, int with_v,
                         DecideArgs D) {
  pdl_enter();
  int slot = blockIdx.z;
  __shared__ double red[2][GX * GY / 32];
  __shared__ int last_blk;
  const int tl = thread_linear();
  if (!slot_running(st, slot)) {
    // a slot that is not cycling still reports "not running"
    if (D.on && D.use_cond && blockIdx.x == 0 && blockIdx.y == 0 && tl == 0)
      report_slot(slot, 0, D.nslot, D.flags, D.counter, D.cond);
    return;
  }
  double r2 = 0.0, v2 = 0.0;
  const int i = blockIdx.x * GX + threadIdx.x;
  const int rows = L.ny * L.nz;
  const int64_t off = (int64_t)(st[slot].k - 1) * col;
  const int tau = st[slot].tau;
  const z64* dg = diag64 ? diag64 + (int64_t)tau * L.n : nullptr;
  const z64* zz = z + slot * vsz + off;
#pragma unroll
  for (int q = 0; q < DEFECT_ROWS; ++q) {
    const int row = (blockIdx.y * DEFECT_ROWS + q) * GY + threadIdx.y;
    if (i >= L.nx || row >= rows) continue;
    const int k = row / L.ny;
    const Cell p{i, row - k * L.ny, k};
    const int c = row * L.nx + i;
    const z64 vv = v[slot * vsv + off + c];
    z64 r = vv;
    if (!zero_z) r = dg ? defect_at(L, p, c, dg[c], vv, zz) : vv - apply_at(L, p, c, taus[tau], zz);
    f0[slot * vsf + c] = cvt<T>(r);
    r2 = fmaT(r.re, r.re, r2);
    r2 = fmaT(r.im, r.im, r2);
    if (with_v) {
      v2 = fmaT(vv.re, vv.re, v2);
      v2 = fmaT(vv.im, vv.im, v2);
    }
  }
  for (int o = 16; o > 0; o >>= 1) r2 += __shfl_down_sync(0xffffffffu, r2, o);
  if (with_v)
    for (int o = 16; o > 0; o >>= 1) v2 += __shfl_down_sync(0xffffffffu, v2, o);
  int w = tl >> 5, lane = tl & 31;
  if (lane == 0) { red[0][w] = r2; red[1][w] = v2; }
  __syncthreads();
  const int nblk = gridDim.x * gridDim.y;
  if (tl == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < GX * GY / 32; ++q) { a += red[0][q]; b += red[1][q]; }
    partial[((int64_t)slot * nblk + block_linear()) * 2 + 0] = a;
    partial[((int64_t)slot * nblk + block_linear()) * 2 + 1] = b;
    if (D.on) {
      __threadfence();
      last_blk = atomicAdd(&D.bcount[slot], 1) == nblk - 1;
    }
  }
  if (!D.on) return;
  __syncthreads();
  if (!last_blk) return;
  __threadfence();
  const double* ps = partial + (int64_t)slot * nblk * 2;
  double a = 0.0, b = 0.0;
  for (int q = tl; q < nblk; q += GX * GY) {
    a += __ldcg(ps + 2 * q);
    b += __ldcg(ps + 2 * q + 1);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  __syncthreads();
  if (lane == 0) { red[0][w] = a; red[1][w] = b; }
  __syncthreads();
  if (tl == 0) {
    a = 0.0;
    b = 0.0;
    for (int q = 0; q < GX * GY / 32; ++q) { a += red[0][q]; b += red[1][q]; }
    D.bcount[slot] = 0;
    int running = decide_slot(st[slot], slot, a, b, zero_z, D.eps, D.max_cycles, D.replay_cycles, D.m_max, D.relax,
                              D.tol);
    if (D.use_cond) report_slot(slot, running, D.nslot, D.flags, D.counter, D.cond);
  }
}

// Sum the per-block partials in a fixed order and decide whether the inner
// solve of each slot is finished; one block per slot. With `use_cond` the last
// block to finish sets the graph's loop condition to "some slot still runs its
// inner solve" (flags[slot] collects the per-slot answers, counter[0] counts
// finished blocks and is reset by the last one).
__global__ void k_inner_decide(SlotState* st, int nslot, const double* __restrict__ partial, int nblocks,
                               int first, double eps, int max_cycles, const int32_t* replay_cycles, int m_max,
                               int use_cond, cudaGraphConditionalHandle cond, int* flags, int* counter, double relax,
                               double tol) {
  __shared__ double red[32];
  int slot = blockIdx.x;
  SlotState& s = st[slot];
  bool act = s.active && !s.inner_done;
  int running = 0;
  if (act) {
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < nblocks; q += blockDim.x) {
      a += partial[((int64_t)slot * nblocks + q) * 2 + 0];
      b += partial[((int64_t)slot * nblocks + q) * 2 + 1];
    }
    a = block_sum(a, red);
    b = block_sum(b, red);
    if (threadIdx.x == 0)
      running = decide_slot(s, slot, a, b, first, eps, max_cycles, replay_cycles, m_max, relax, tol);
  }
  if (use_cond && threadIdx.x == 0) report_slot(slot, running, nslot, flags, counter, cond);
}

// K_cc + tau_q M_cc for every distinct tau in fp64 (the diagonal apply_at forms).
__global__ void k_diag64(LevelView<double> L, const z64* __restrict__ taus, int ntau, z64* __restrict__ out) {
  Cell p;
  int c;
  if (!grid_cell(L.nx, L.ny, L.nz, &p, &c)) return;
  const double d = L.kd ? L.kd[c] : fsum(faces_at(L, p));
  const double m = L.mm[c];
  for (int q = 0; q < ntau; ++q) out[(int64_t)q * L.n + c] = mk(fmaT(taus[q].re, m, d), mulT(taus[q].im, m));
}

// K diagonal (sum of each cell's faces), the same sum apply_at forms.
__global__ void k_kdiag(LevelView<double> L, double* __restrict__ kd) {
  Cell p;
  int c;
  if (!grid_cell(L.nx, L.ny, L.nz, &p, &c)) return;
  kd[c] = fsum(faces_at(L, p));
}

// --------------------------------------------------------------------- launchers
static inline unsigned nb(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }
static inline dim3 grid2(int64_t nxw, int64_t rows, int nz) { return dim3(nb(nxw, GX), nb(rows, GY), nz); }
static const dim3 B2(GX, GY);

void launch_faces_from_cond(const LevelHost& L, const double h[3], uint32_t mask, const double* cond,
                            cudaStream_t s) {
  int64_t tot = face_count(L, 0) + face_count(L, 1) + (L.nz > 1 ? face_count(L, 2) : 0);
  k_faces_from_cond<<<nb(tot, 256), 256, 0, s>>>(L.nx, L.ny, L.nz, h[0], h[1], h[2], mask, cond, L.d64[0],
                                                  L.d64[1], L.d64[2]);
}

void launch_coarsen(const LevelHost& F, const LevelHost& C, const double* fac_x, const double* fac_y,
                    const double* fac_z, cudaStream_t s) {
  int64_t tot = face_count(C, 0) + face_count(C, 1) + (C.nz > 1 || F.nz > 1 ? face_count(C, 2) : 0) + C.n;
  k_coarsen<<<nb(tot, 256), 256, 0, s>>>(view<double>(F), F.rx, F.ry, F.rz, C.nx, C.ny, C.nz, C.d64[0], C.d64[1],
                                          C.d64[2], C.d64[3], fac_x, fac_y, fac_z);
}

std::vector<double> coarse_face_factors(const std::vector<double>& w, int r, std::vector<double>* W) {
  const int n = (int)w.size();
  if (r == 1) {
    *W = w;
    return std::vector<double>(n + 1, 1.0);
  }
  const int nc = (n + 1) / 2;
  W->assign(nc, 0.0);
  for (int I = 0; I < nc; ++I) (*W)[I] = w[2 * I] + (2 * I + 1 < n ? w[2 * I + 1] : 0.0);
  std::vector<double> f(nc + 1);
  f[0] = w[0] / (*W)[0];
  for (int I = 1; I < nc; ++I) f[I] = (w[2 * I - 1] + w[2 * I]) / ((*W)[I - 1] + (*W)[I]);
  f[nc] = w[n - 1] / (*W)[nc - 1];
  return f;
}

void launch_to_f32(const double* a, float* b, int64_t n, cudaStream_t s) {
  k_to_f32<<<nb(n, 256), 256, 0, s>>>(a, b, n);
}

template <typename T>
void launch_invd(const LevelHost& L, const z64* taus, int ntau, cx<T>* out, cudaStream_t s, int from_f32) {
  if (from_f32) k_invd<T, float><<<nb(L.n, 256), 256, 0, s>>>(view_as<double, float>(L), taus, ntau, out);
  else k_invd<T, double><<<nb(L.n, 256), 256, 0, s>>>(view<double>(L), taus, ntau, out);
}

void launch_coarse_inverse(const LevelHost& L, const z64* taus, int ntau, z64* work, z64* inv, int* singular,
                           cudaStream_t s, int from_f32) {
  if (from_f32) k_coarse_dense<float><<<nb(L.n, 128), 128, 0, s>>>(view_as<double, float>(L), taus, ntau, work);
  else k_coarse_dense<double><<<nb(L.n, 128), 128, 0, s>>>(view<double>(L), taus, ntau, work);
  k_gauss_jordan<<<ntau, 1024, 0, s>>>(work, inv, (int)L.n, singular);
}

void launch_round_bf16(const double* a, __nv_bfloat16* b, float* r, int64_t n, cudaStream_t s) {
  k_round_bf16<<<nb(n, 256), 256, 0, s>>>(a, b, r, n);
}

template <typename T>
void launch_to_prec(const z64* a, cx<T>* b, int64_t n, cudaStream_t s) {
  k_to_prec<T><<<nb(n, 256), 256, 0, s>>>(a, b, n);
}

template <typename T>
void launch_apply(const LevelHost& L, z64 sfix, const SlotState* st, const z64* taus, const cx<T>* x, cx<T>* y,
                  int64_t vs, int nslot, cudaStream_t s) {
  k_apply<T><<<grid2(L.nx, (int64_t)L.ny * L.nz, nslot), B2, 0, s>>>(view<T>(L), sfix, st, taus, x, y, vs);
}

// Sources per block of the multi-source smoother and restriction: a power of
// two up to 8 (blockDim = (32, 8 / G, G)).
static int spmm_group(int nslot) {
  int g = 1;
  while (g < 8 && 2 * g <= nslot) g *= 2;
  return g;
}

template <typename T>
void launch_gs(const LevelHost& L, const SlotState* st, const cx<T>* invd, const cx<T>* f, cx<T>* z, int64_t vs,
               int nslot, int color, int zero_start, cudaStream_t s, z64* Zk, int64_t vsZk, int64_t zcol, int bf16) {
  const int G = spmm_group(nslot), rb = GY / G;
  const dim3 blk(GX, rb, G), grd(nb((L.nx + 1) / 2, GX), nb((int64_t)L.ny * L.nz, rb), nb(nslot, G));
  if constexpr (sizeof(T) == 4) {
    if (bf16) {
      if (Zk)
        launch_pdl(k_gs_correct<T, __nv_bfloat16>, grd, blk, 0, s, view_as<T, __nv_bfloat16>(L), st, invd, f, z, vs, color,
                                                           Zk, vsZk, zcol, nslot);
      else
        launch_pdl(k_gs<T, __nv_bfloat16>, grd, blk, 0, s, view_as<T, __nv_bfloat16>(L), st, invd, f, z, vs, color,
                                                   zero_start, nslot);
      return;
    }
  }
  if (Zk) {
    launch_pdl(k_gs_correct<T, T>, grd, blk, 0, s, view<T>(L), st, invd, f, z, vs, color, Zk, vsZk, zcol, nslot);
    return;
  }
  launch_pdl(k_gs<T, T>, grd, blk, 0, s, view<T>(L), st, invd, f, z, vs, color, zero_start, nslot);
}

template <typename T>
void launch_residual_restrict(const LevelHost& F, const LevelHost& C, const SlotState* st, const z64* taus,
                              const cx<T>* f, const cx<T>* z, int64_t vs, cx<T>* fc, int64_t vsc, int nslot,
                              cudaStream_t s, int bf16) {
  const int G = spmm_group(nslot), rb = GY / G;
  if (G == 1 && F.nz > 1 && F.rx == 2 && F.ry == 2 && F.rz == 2 && (int64_t)nb(F.ny, GY) * C.nz <= 65535) {
    // one source: the tile form (with several, the per-coarse-cell form reads
    // each coefficient once for the block's sources)
    const dim3 g3(nb(F.nx, GX), nb(F.ny, GY) * C.nz, nslot);
    if constexpr (sizeof(T) == 4) {
      if (bf16) {
        launch_pdl(k_residual_restrict3<T, __nv_bfloat16>, g3, B2, 0, s, view_as<T, __nv_bfloat16>(F), C.nx, C.ny,
                   C.nz, st, taus, f, z, vs, fc, vsc);
        return;
      }
    }
    launch_pdl(k_residual_restrict3<T, T>, g3, B2, 0, s, view<T>(F), C.nx, C.ny, C.nz, st, taus, f, z, vs, fc, vsc);
    return;
  }
  const dim3 blk(GX, rb, G), grd(nb(C.nx, GX), nb((int64_t)C.ny * C.nz, rb), nb(nslot, G));
  if constexpr (sizeof(T) == 4) {
    if (bf16) {
      launch_pdl(k_residual_restrict<T, __nv_bfloat16>, grd, blk, 0, s, view_as<T, __nv_bfloat16>(F), F.rx, F.ry, F.rz, C.nx,
                                                                C.ny, C.nz, st, taus, f, z, vs, fc, vsc, nslot);
      return;
    }
  }
  launch_pdl(k_residual_restrict<T, T>, grd, blk, 0, s, view<T>(F), F.rx, F.ry, F.rz, C.nx, C.ny, C.nz, st, taus, f, z, vs, fc,
                                                vsc, nslot);
}

template <typename T>
void launch_prolong_add(const LevelHost& F, const LevelHost& C, uint32_t mask, const SlotState* st, const cx<T>* zc,
                        int64_t vsc, cx<T>* z, int64_t vs, int nslot, cudaStream_t s) {
  if (F.nz > 1 && F.rx == 2 && F.ry == 2 && F.rz == 2 && (int64_t)nb(F.ny, GY) * C.nz <= 65535) {
    const dim3 g(nb(F.nx, GX), nb(F.ny, GY) * C.nz, nslot);
    launch_pdl(k_prolong_add3<T>, g, B2, 0, s, view<T>(F), C.nx, C.ny, C.nz, mask, st, zc, vsc, z, vs);
    return;
  }
  launch_pdl(k_prolong_add<T>, grid2(F.nx, (int64_t)F.ny * F.nz, nslot), B2, 0, s, view<T>(F), F.rx, F.ry, F.rz, C.nx, C.ny,
                                                                            C.nz, mask, st, zc, vsc, z, vs);
}

// Tiles of 32x32 or 16x16 cells (16x16: more blocks on small grids, a larger
// share of recomputed halo); the caller picks per level.
template <typename T, int TX, int TY>
static size_t fused_smem() {
  return 2 * (size_t)(TX + 2 * FH) * (TY + 2 * FH) * sizeof(cx<T>);
}

bool fused_level_ok(const LevelHost& L) {
  return L.nz == 1 && L.rx == 2 && L.ry == 2 && L.rz == 1 && L.nx % 2 == 0 && L.ny % 2 == 0;
}

template <typename T>
void fused_prepare() {
  // 8 x 8 and 16 x 16 tiles stay under the 48 KB default
  cudaFuncSetAttribute(k_pre2d<T, 32, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem<T, 32, 32>());
  cudaFuncSetAttribute(k_post2d<T, 32, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem<T, 32, 32>());
}

template <typename T>
void launch_pre2d(const LevelHost& F, const LevelHost& C, const SlotState* st, const cx<T>* invd, const z64* taus,
                  const cx<T>* f, cx<T>* z, int64_t vs, cx<T>* fc, int64_t vsc, int nslot, int tile, cudaStream_t s) {
  if (tile == 8) {
    dim3 g(nb(F.nx, 8), nb(F.ny, 8), nslot);
    launch_pdl(k_pre2d<T, 8, 8>, g, 256, fused_smem<T, 8, 8>(), s, view<T>(F), st, invd, taus, f, z, vs, fc, vsc);
  } else if (tile == 16) {
    dim3 g(nb(F.nx, 16), nb(F.ny, 16), nslot);
    launch_pdl(k_pre2d<T, 16, 16>, g, 256, fused_smem<T, 16, 16>(), s, view<T>(F), st, invd, taus, f, z, vs, fc, vsc);
  } else {
    dim3 g(nb(F.nx, 32), nb(F.ny, 32), nslot);
    launch_pdl(k_pre2d<T, 32, 32>, g, 256, fused_smem<T, 32, 32>(), s, view<T>(F), st, invd, taus, f, z, vs, fc, vsc);
  }
  (void)C;
}

template <typename T>
void launch_post2d(const LevelHost& F, const LevelHost& C, uint32_t mask, const SlotState* st, const cx<T>* invd,
                   const cx<T>* f, const cx<T>* z, cx<T>* zout, int64_t vs, const cx<T>* zc, int64_t vsc, int nslot,
                   int tile, cudaStream_t s, z64* Zk, int64_t vsZk, int64_t zcol) {
  if (tile == 8) {
    dim3 g(nb(F.nx, 8), nb(F.ny, 8), nslot);
    launch_pdl(k_post2d<T, 8, 8>, g, 256, fused_smem<T, 8, 8>(), s, view<T>(F), mask, st, invd, f, z, zout, vs, zc, vsc, Zk,
                                                             vsZk, zcol);
  } else if (tile == 16) {
    dim3 g(nb(F.nx, 16), nb(F.ny, 16), nslot);
    launch_pdl(k_post2d<T, 16, 16>, g, 256, fused_smem<T, 16, 16>(), s, view<T>(F), mask, st, invd, f, z, zout, vs, zc, vsc,
                                                                 Zk, vsZk, zcol);
  } else {
    dim3 g(nb(F.nx, 32), nb(F.ny, 32), nslot);
    launch_pdl(k_post2d<T, 32, 32>, g, 256, fused_smem<T, 32, 32>(), s, view<T>(F), mask, st, invd, f, z, zout, vs, zc, vsc,
                                                                 Zk, vsZk, zcol);
  }
  (void)C;
}

template <typename T>
void tail_prepare(size_t smem_bytes) {
  cudaFuncSetAttribute(k_tail_vcycle<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  cudaFuncSetAttribute(k_tail2d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

template <typename T>
void launch_tail(const TailParams<T>& P, size_t smem_bytes, const SlotState* st, int nslot, cudaStream_t s) {
  if (P.pairs)
    launch_pdl(k_tail2d<T>, nslot, TAIL_THREADS, smem_bytes, s, P, st);
  else
    launch_pdl(k_tail_vcycle<T>, nslot, TAIL_THREADS, smem_bytes, s, P, st);
}

template <typename T>
void launch_coarse_solve(const cx<T>* Ainv, int n, const SlotState* st, const cx<T>* f, cx<T>* z, int64_t vs,
                         int nslot, cudaStream_t s) {
  dim3 g(nb(n, 128), nslot);
  k_coarse_solve<T><<<g, 128, 0, s>>>(Ainv, n, st, f, z, vs);
}

template <typename T>
void launch_correct(const SlotState* st, z64* z, int64_t zs, int64_t zcol, const cx<T>* e, int64_t es, int64_t n,
                    int nslot, cudaStream_t s) {
  dim3 g(nb(n, 256), nslot);
  k_correct<T><<<g, 256, 0, s>>>(st, z, zs, zcol, e, es, n);
}

static dim3 defect_grid(const LevelHost& L, int nslot) {
  return dim3(nb(L.nx, GX), nb((int64_t)L.ny * L.nz, GY * DEFECT_ROWS), nslot);
}

int defect_blocks(const LevelHost& L) {
  dim3 g = defect_grid(L, 1);
  return (int)(g.x * g.y);
}

template <typename T>
void launch_defect(const LevelHost& L, const SlotState* st, const z64* taus, const z64* v, int64_t vsv, const z64* z,
                   int64_t vsz, int64_t col, int zero_z, cx<T>* f0, int64_t vsf, double* partial, int with_v,
                   int nslot, cudaStream_t s) {
  DecideArgs D{};
  launch_pdl(k_defect<T>, defect_grid(L, nslot), B2, 0, s, view<double>(L), const_cast<SlotState*>(st), taus, nullptr, v, vsv,
                                                   z, vsz, col, zero_z, f0, vsf, partial, with_v, D);
}

template <typename T>
void launch_defect_decide(const LevelHost& L, SlotState* st, const z64* taus, const z64* diag64, const z64* v,
                          int64_t vsv, const z64* z, int64_t vsz, int64_t col, int zero_z, cx<T>* f0, int64_t vsf,
                          double* partial, double eps, int max_cycles, const int32_t* replay_cycles, int m_max,
                          int use_cond, cudaGraphConditionalHandle cond, int* flags, int* counter, int* bcount,
                          int nslot, double relax, double tol, cudaStream_t s) {
  DecideArgs D{1, eps, max_cycles, replay_cycles, m_max, use_cond, cond, flags, counter, bcount, nslot, relax, tol};
  launch_pdl(k_defect<T>, defect_grid(L, nslot), B2, 0, s, view<double>(L), st, taus, diag64, v, vsv, z, vsz, col, zero_z,
                                                   f0, vsf, partial, zero_z, D);
}

void launch_diag64(const LevelHost& L, const z64* taus, int ntau, z64* out, cudaStream_t s) {
  k_diag64<<<grid2(L.nx, (int64_t)L.ny * L.nz, 1), B2, 0, s>>>(view<double>(L), taus, ntau, out);
}

void launch_kdiag(const LevelHost& L, double* kd, cudaStream_t s) {
  k_kdiag<<<grid2(L.nx, (int64_t)L.ny * L.nz, 1), B2, 0, s>>>(view<double>(L), kd);
}

void launch_inner_decide(SlotState* st, int nslot, const double* partial, int nblocks, int first, double eps,
                         int max_cycles, const int32_t* replay_cycles, int m_max, int use_cond,
                         cudaGraphConditionalHandle cond, int* flags, int* counter, cudaStream_t s, double relax,
                         double tol) {
  k_inner_decide<<<nslot, 512, 0, s>>>(st, nslot, partial, nblocks, first, eps, max_cycles, replay_cycles, m_max,
                                        use_cond, cond, flags, counter, relax, tol);
}

#define INST(T)                                                                                                  \
  template void fused_prepare<T>();                                                                               \
  template void launch_pre2d<T>(const LevelHost&, const LevelHost&, const SlotState*, const cx<T>*, const z64*,    \
                                const cx<T>*, cx<T>*, int64_t, cx<T>*, int64_t, int, int, cudaStream_t);          \
  template void launch_post2d<T>(const LevelHost&, const LevelHost&, uint32_t, const SlotState*, const cx<T>*,     \
                                 const cx<T>*, const cx<T>*, cx<T>*, int64_t, const cx<T>*, int64_t, int, int,    \
                                 cudaStream_t, z64*, int64_t, int64_t);                                           \
  template void tail_prepare<T>(size_t);                                                                          \
  template void launch_tail<T>(const TailParams<T>&, size_t, const SlotState*, int, cudaStream_t);                \
  template void launch_invd<T>(const LevelHost&, const z64*, int, cx<T>*, cudaStream_t, int);                     \
  template void launch_to_prec<T>(const z64*, cx<T>*, int64_t, cudaStream_t);                                     \
  template void launch_apply<T>(const LevelHost&, z64, const SlotState*, const z64*, const cx<T>*, cx<T>*, int64_t, \
                                int, cudaStream_t);                                                               \
  template void launch_gs<T>(const LevelHost&, const SlotState*, const cx<T>*, const cx<T>*, cx<T>*, int64_t, int,  \
                             int, int, cudaStream_t, z64*, int64_t, int64_t, int);                                \
  template void launch_residual_restrict<T>(const LevelHost&, const LevelHost&, const SlotState*, const z64*,      \
                                            const cx<T>*, const cx<T>*, int64_t, cx<T>*, int64_t, int,           \
                                            cudaStream_t, int);                                                   \
  template void launch_prolong_add<T>(const LevelHost&, const LevelHost&, uint32_t, const SlotState*,             \
                                      const cx<T>*, int64_t, cx<T>*, int64_t, int, cudaStream_t);                 \
  template void launch_coarse_solve<T>(const cx<T>*, int, const SlotState*, const cx<T>*, cx<T>*, int64_t, int,    \
                                       cudaStream_t);                                                             \
  template void launch_correct<T>(const SlotState*, z64*, int64_t, int64_t, const cx<T>*, int64_t, int64_t, int,  \
                                  cudaStream_t);                                                                  \
  template void launch_defect<T>(const LevelHost&, const SlotState*, const z64*, const z64*, int64_t, const z64*,  \
                                 int64_t, int64_t, int, cx<T>*, int64_t, double*, int, int, cudaStream_t);       \
  template void launch_defect_decide<T>(const LevelHost&, SlotState*, const z64*, const z64*, const z64*, int64_t, \
                                        const z64*, int64_t, int64_t, int, cx<T>*, int64_t, double*, double, int, \
                                        const int32_t*, int, int, cudaGraphConditionalHandle, int*, int*, int*, int, \
                                        double, double, cudaStream_t);

INST(double)
INST(float)

}  // namespace fks
