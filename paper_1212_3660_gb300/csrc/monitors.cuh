// Prop. 1's Ritz values on the GPU (monitors.cu).
#pragma once
#include "common.cuh"

namespace fks {

// theta [n_rhs][m_max]: the eigenvalues of H_m^{-1} - T_m of every source
// (m = steps[r]; zero beyond m), from hbar [n_rhs][(m_max + 1) m_max]
// (column-major) and tau_k [n_rhs][m_max]; status [n_rhs]: 0 converged,
// 1 sweep limit reached (theta then holds the unconverged diagonal),
// 2 H_m singular. scratch: 2 n_rhs m_max^2 complex.
void launch_ritz(const z64* hbar, const z64* tau_k, const int32_t* steps, int n_rhs, int m_max, z64* scratch,
                 z64* theta, int32_t* status, cudaStream_t s);

}  // namespace fks
