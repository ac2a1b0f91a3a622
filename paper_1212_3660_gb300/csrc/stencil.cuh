// Device helpers for the cell-centred 2d+1-point operator, shared by the grid
// and Krylov kernels.
#pragma once
#include "common.cuh"

namespace fks {

// --------------------------------------------------------------------- indexing
struct Cell {
  int i, j, k;
};

// Cell of flat index c (32-bit: a level has fewer than 2^31 cells).
__device__ __forceinline__ Cell cell_of(int c, int nx, int ny) {
  Cell r;
  int q = c / nx;
  r.i = c - q * nx;
  r.k = q / ny;
  r.j = q - r.k * ny;
  return r;
}

// Launch shape of the grid kernels: block (GX, GY) threads, x along i, y along
// the rows (j, k) of the level, z along the sources.
constexpr int GX = 32, GY = 8;

// Cell of this thread in a (i, row) launch; false past the grid.
__device__ __forceinline__ bool grid_cell(int nx, int ny, int nz, Cell* p, int* c) {
  int i = blockIdx.x * GX + threadIdx.x;
  int row = blockIdx.y * GY + threadIdx.y;
  if (i >= nx || row >= ny * nz) return false;
  int k = row / ny;
  *p = Cell{i, row - k * ny, k};
  *c = row * nx + i;
  return true;
}

// Cell of colour `color` of this thread in a (half-row index, row) launch.
__device__ __forceinline__ bool grid_color_cell(int nx, int ny, int nz, int color, Cell* p, int* c) {
  int ii = blockIdx.x * GX + threadIdx.x;
  int row = blockIdx.y * GY + threadIdx.y;
  if (row >= ny * nz) return false;
  int k = row / ny;
  int j = row - k * ny;
  int i = 2 * ii + ((j + k + color) & 1);
  if (i >= nx) return false;
  *p = Cell{i, j, k};
  *c = row * nx + i;
  return true;
}

__device__ __forceinline__ int block_linear() { return blockIdx.y * gridDim.x + blockIdx.x; }
__device__ __forceinline__ int thread_linear() { return threadIdx.y * GX + threadIdx.x; }

template <typename T>
struct Faces {
  T xl, xh, yl, yh, zl, zh;
};

template <typename T, typename C>
__device__ __forceinline__ Faces<T> faces_at(const LevelView<T, C>& L, Cell p) {
  Faces<T> f;
  int64_t rx = ((int64_t)p.k * L.ny + p.j) * (L.nx + 1) + p.i;
  f.xl = ldc<T>(L.fx, rx);
  f.xh = ldc<T>(L.fx, rx + 1);
  int64_t ry = ((int64_t)p.k * (L.ny + 1) + p.j) * L.nx + p.i;
  f.yl = ldc<T>(L.fy, ry);
  f.yh = ldc<T>(L.fy, ry + L.nx);
  if (L.nz > 1) {
    int64_t rz = ((int64_t)p.k * L.ny + p.j) * L.nx + p.i;
    f.zl = ldc<T>(L.fz, rz);
    f.zh = ldc<T>(L.fz, rz + (int64_t)L.nx * L.ny);
  } else {
    f.zl = T(0);
    f.zh = T(0);
  }
  return f;
}

template <typename T>
__device__ __forceinline__ T fsum(const Faces<T>& f) {
  return ((f.xl + f.xh) + (f.yl + f.yh)) + (f.zl + f.zh);
}

// s0 + sum over existing neighbours of t_face * x_nb (accumulated in this order)
template <typename T, typename C>
__device__ __forceinline__ cx<T> nb_sum(const LevelView<T, C>& L, const Faces<T>& f, Cell p, int64_t c,
                                        const cx<T>* __restrict__ x, cx<T> s0 = cx<T>{T(0), T(0)}) {
  cx<T> s = s0;
  int64_t sxy = (int64_t)L.nx * L.ny;
  if (p.i > 0) s = axpy(f.xl, x[c - 1], s);
  if (p.i < L.nx - 1) s = axpy(f.xh, x[c + 1], s);
  if (p.j > 0) s = axpy(f.yl, x[c - L.nx], s);
  if (p.j < L.ny - 1) s = axpy(f.yh, x[c + L.nx], s);
  if (L.nz > 1) {
    if (p.k > 0) s = axpy(f.zl, x[c - sxy], s);
    if (p.k < L.nz - 1) s = axpy(f.zh, x[c + sxy], s);
  }
  return s;
}

template <typename T, typename C>
__device__ __forceinline__ cx<T> apply_at(const LevelView<T, C>& L, Cell p, int64_t c, cx<T> s,
                                          const cx<T>* __restrict__ x) {
  Faces<T> f = faces_at(L, p);
  T d = L.kd ? L.kd[c] : fsum(f);  // same sum either way
  T m = ldc<T>(L.mm, c);
  cx<T> diag = mk(fmaT(s.re, m, d), mulT(s.im, m));
  return diag * x[c] - nb_sum(L, f, p, c, x);
}

// v_c - ((K + tau M) x)_c with diag = K_cc + tau M_cc given: the neighbour
// terms accumulate onto v, then diag * x_c is subtracted with fused
// multiply-adds (fewer FP64 operations than v - apply_at).
template <typename T, typename C>
__device__ __forceinline__ cx<T> defect_at(const LevelView<T, C>& L, Cell p, int64_t c, cx<T> diag, cx<T> v,
                                           const cx<T>* __restrict__ x) {
  Faces<T> f = faces_at(L, p);
  cx<T> acc = nb_sum(L, f, p, c, x, v);
  const cx<T> xc = x[c];
  acc.re = fmaT(-diag.re, xc.re, fmaT(diag.im, xc.im, acc.re));
  acc.im = fmaT(-diag.re, xc.im, fmaT(-diag.im, xc.re, acc.im));
  return acc;
}

// Red-black Gauss-Seidel update of cell c: (f_c + sum_nb t z_nb) / (K_cc + tau M_cc),
// the neighbours taken as zero when `zero_start`.
template <typename T, typename C>
__device__ __forceinline__ cx<T> gs_value(const LevelView<T, C>& L, Cell p, int64_t c, cx<T> id, const cx<T>* f,
                                          const cx<T>* z, int zero_start) {
  cx<T> rhs = f[c];
  if (!zero_start) {
    Faces<T> fc = faces_at(L, p);
    rhs = nb_sum(L, fc, p, c, z, rhs);  // f + sum t z_nb, accumulated from f
  }
  return id * rhs;
}

// Cell of colour `color` handled by work item t of a half sweep (false if none).
__device__ __forceinline__ bool color_cell(int nx, int ny, int nz, int color, int t, Cell* p, int* c) {
  int nxh = (nx + 1) >> 1;
  int rows = ny * nz;
  if (t >= nxh * rows) return false;
  int row = t / nxh;
  int k = row / ny;
  int j = row - k * ny;
  int i = 2 * (t - row * nxh) + ((j + k + color) & 1);
  if (i >= nx) return false;
  *p = Cell{i, j, k};
  *c = row * nx + i;
  return true;
}

// Sum over the children of coarse cell (I,J,K) of the fine residual f - (K + s M) z
// (on an odd axis the last coarse cell has one child).
template <typename T, typename C>
__device__ __forceinline__ cx<T> restrict_value(const LevelView<T, C>& F, int rx, int ry, int rz, int I, int J, int K,
                                                cx<T> s, const cx<T>* f, const cx<T>* z) {
  cx<T> acc = mk(T(0), T(0));
  for (int c = 0; c < rz; ++c)
    for (int b = 0; b < ry; ++b)
      for (int a = 0; a < rx; ++a) {
        Cell p{rx * I + a, ry * J + b, rz * K + c};
        if (p.i >= F.nx || p.j >= F.ny || p.k >= F.nz) continue;
        int64_t cc = ((int64_t)p.k * F.ny + p.j) * F.nx + p.i;
        acc = acc + (f[cc] - apply_at(F, p, cc, s, z));
      }
  return acc;
}

// (P zc)_c: cell-centred (bi/tri)linear interpolation from the coarser level.
// Per coarsened axis: 3/4 on the parent, 1/4 on the coarse neighbour on the
// child's side; past a zero-head face the ghost is -parent (weight 1/2 on the
// parent), past a no-flow face +parent (weight 1).
// get(X, Y, Z) returns the coarse value at coarse cell (X, Y, Z).
template <typename T, typename Get>
__device__ __forceinline__ cx<T> prolong_value_at(Cell p, int rx, int ry, int rz, int cnx, int cny, int cnz,
                                                  uint32_t mask, Get get) {
  int par[3] = {p.i / rx, p.j / ry, p.k / rz};
  int idx[3] = {p.i, p.j, p.k};
  int rr[3] = {rx, ry, rz};
  int nn[3] = {cnx, cny, cnz};
  int ti[3][2];
  T tw[3][2];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ti[a][0] = par[a];
    ti[a][1] = par[a];
    if (rr[a] == 1) {
      tw[a][0] = T(1);
      tw[a][1] = T(0);
      continue;
    }
    int nb = (idx[a] & 1) ? par[a] + 1 : par[a] - 1;
    if (nb >= 0 && nb < nn[a]) {
      tw[a][0] = T(0.75);
      ti[a][1] = nb;
      tw[a][1] = T(0.25);
    } else {
      bool dir = nb < 0 ? ((mask >> (2 * a)) & 1u) : ((mask >> (2 * a + 1)) & 1u);
      tw[a][0] = dir ? T(0.5) : T(1);
      tw[a][1] = T(0);
    }
  }
  cx<T> acc = mk(T(0), T(0));
#pragma unroll
  for (int c2 = 0; c2 < 2; ++c2) {
    T wz = tw[2][c2];
    if (wz == T(0)) continue;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      T wy = tw[1][b];
      if (wy == T(0)) continue;
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        T wx = tw[0][a];
        if (wx == T(0)) continue;
        acc = axpy(mulT(mulT(wx, wy), wz), get(ti[0][a], ti[1][b], ti[2][c2]), acc);
      }
    }
  }
  return acc;
}

template <typename T>
__device__ __forceinline__ cx<T> prolong_value(Cell p, int rx, int ry, int rz, int cnx, int cny, int cnz,
                                               uint32_t mask, const cx<T>* zc) {
  return prolong_value_at<T>(p, rx, ry, rz, cnx, cny, cnz, mask, [&](int X, int Y, int Z) {
    return zc[((int64_t)Z * cny + Y) * cnx + X];
  });
}

}  // namespace fks
