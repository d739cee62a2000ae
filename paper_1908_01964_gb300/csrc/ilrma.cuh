// Internal declarations of the initialisation from the outputs of the ILRMA
// stage (rcscm_ilrma_init; kernels in ilrma.cu).
#pragma once

#include "rcscm_internal.cuh"

namespace rcscm {

// One utterance of rcscm_ilrma_init (device views of the caller's buffers).
struct IlrmaArgs {
    int I, J, M, K, n_h;
    const float2* x;       // [I][J][M]
    const double2* W;      // [I][M][M], row n = w_{i,n}^H
    const float* T;        // [I][K]
    const float* V;        // [K][J]
    double2* a;            // [I][M]
    double2* Rp;           // [I][M][M]
    float* rh0;            // [I][J]
    float* ru0;            // [I][J]
};
constexpr int kIlrmaMaxK = 256;   // NMF bases per source held in shared memory
cudaError_t launch_ilrma_init(const IlrmaArgs& u, int* status, cudaStream_t s);

}  // namespace rcscm
