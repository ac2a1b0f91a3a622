// Sensitivities of the phasor measurements by the adjoint-state method
// (Section 5, Eq. sensitivity with the adjoint of Eq. adjoint, Algorithm 6), in
// the cell-centred discretisation: with A = K + sigma M, A Phi = b, h = Phi(x_m)
// and A Psi = -e_m (A is complex symmetric, so the adjoint operator is A),
//   dh/dp = Psi^T (dA/dp) Phi.
// For p = ln S_s,c:  sigma M_cc Psi_c Phi_c.
// For p = ln K_c, over the faces of cell c (transmissibility t):
//   interior face to nb:  t K_nb / (K_c + K_nb) (Psi_c - Psi_nb)(Phi_c - Phi_nb)
//     (t = g 2 K_c K_nb / (K_c + K_nb), so dt/dlnK_c = t K_nb / (K_c + K_nb))
//   zero-head boundary face: t Psi_c Phi_c  (t = 2 g K_c; no-flow faces carry t = 0)
// One thread per cell and shift: Phi's neighbourhood, the faces and the
// conductivities are loaded and folded into one complex weight per face once,
// then the measurements are looped over. On GB300 the kernel is bound by FP64
// arithmetic (per cell, shift and measurement: 2 subtractions and 4 fused
// multiply-adds per face and a complex product), not by memory.
#include "sensitivity.cuh"
#include "stencil.cuh"

namespace fks {

constexpr int SENS_THREADS = 256;

__global__ void __launch_bounds__(SENS_THREADS) k_sensitivity(LevelView<double> L, const double* __restrict__ cond,
                                                              const z64* __restrict__ phi, const z64* __restrict__ psi,
                                                              int n_m, int n_f, const z64* __restrict__ sigma,
                                                              z64* __restrict__ jk, z64* __restrict__ js) {
  const int64_t c = (int64_t)blockIdx.x * SENS_THREADS + threadIdx.x;
  const int j = blockIdx.y;
  if (c >= L.n) return;
  const Cell p = cell_of((int)c, L.nx, L.ny);
  const Faces<double> f = faces_at(L, p);
  const double kc = cond[c];
  const int64_t sxy = (int64_t)L.nx * L.ny;
  // per face: neighbour offset (0: boundary face) and a_f = (dt/dlnK_c)(Phi_c - Phi_nb)
  // (boundary face: (dt/dlnK_c) Phi_c), reused for every measurement
  const int nfaces = L.nz > 1 ? 6 : 4;
  int64_t off[6];
  z64 af[6];
  const double t[6] = {f.xl, f.xh, f.yl, f.yh, f.zl, f.zh};
  const bool inner[6] = {p.i > 0, p.i < L.nx - 1, p.j > 0, p.j < L.ny - 1, p.k > 0, p.k < L.nz - 1};
  const int64_t step[6] = {-1, 1, -(int64_t)L.nx, (int64_t)L.nx, -sxy, sxy};
  const z64* ph = phi + (int64_t)j * L.n;
  const z64 phc = ph[c];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    off[a] = 0;
    af[a] = mk(0.0, 0.0);
    if (a >= nfaces) continue;
    if (inner[a]) {
      off[a] = step[a];
      const double kn = cond[c + step[a]];
      af[a] = (t[a] * (kn / (kc + kn))) * (phc - ph[c + step[a]]);
    } else {
      af[a] = t[a] * phc;
    }
  }
  const z64 smphi = (L.mm[c] * sigma[j]) * phc;  // sigma M_cc Phi_c
  for (int m = 0; m < n_m; ++m) {
    const int64_t base = ((int64_t)m * n_f + j) * L.n;
    const z64* ps = psi + base;
    const z64 psc = ps[c];
    z64 acc = mk(0.0, 0.0);
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      if (a >= nfaces) continue;
      const z64 dpsi = off[a] ? psc - ps[c + off[a]] : psc;
      // acc += dpsi * a_f in four fused multiply-adds
      acc.re = fmaT(dpsi.re, af[a].re, fmaT(-dpsi.im, af[a].im, acc.re));
      acc.im = fmaT(dpsi.re, af[a].im, fmaT(dpsi.im, af[a].re, acc.im));
    }
    jk[base + c] = acc;
    js[base + c] = smphi * psc;
  }
}

void launch_sensitivity(const LevelHost& L0, const double* cond, const z64* phi, const z64* psi, int n_m, int n_f,
                        const z64* sigma, z64* jk, z64* js, cudaStream_t s) {
  const dim3 g((unsigned)((L0.n + SENS_THREADS - 1) / SENS_THREADS), (unsigned)n_f);
  k_sensitivity<<<g, SENS_THREADS, 0, s>>>(view<double>(L0), cond, phi, psi, n_m, n_f, sigma, jk, js);
}

}  // namespace fks
