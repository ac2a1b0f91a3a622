// Adjoint-state sensitivities of the phasor measurements (sensitivity.cu).
#pragma once
#include "common.cuh"

namespace fks {

// jk, js [n_m][n_f][n]: dh/dlnK_c and dh/dlnS_c of measurement m at shift j,
// from the forward phasors phi [n_f][n], the adjoint phasors psi [n_m][n_f][n],
// the shifts sigma [n_f] and the cell conductivities cond [n] of level L0.
void launch_sensitivity(const LevelHost& L0, const double* cond, const z64* phi, const z64* psi, int n_m, int n_f,
                        const z64* sigma, z64* jk, z64* js, cudaStream_t s);

}  // namespace fks
