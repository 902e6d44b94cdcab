// Tensor-core emissivity: parameters and launchers (k_emis_tc.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

namespace heat {

constexpr int kMaxTcGrains = 96;  // grains per launch (tensor maps travel as kernel parameters)

struct EmisTcParams {
    CUtensorMap ta[kMaxTcGrains];  // A'_g: [cells][Kp_g] operand, 128B swizzle, box 128 rows
    CUtensorMap tb[kMaxTcGrains];  // B'_g: [N][Kp_g] operand, box ntile rows (256 or 128)
    int ksteps[kMaxTcGrains];      // k blocks: (split ? Kp_g / 2 : Kp_g) / elements per 128-byte slice
    int grain[kMaxTcGrains];       // grain index of slot i
    int ng;                        // grains in this launch
    int cells, N, G;
    int mtiles, ntiles;            // ceil(cells/128), ceil(N/256)
    const float* rowscale;         // [cells][G] power-of-two scale of A'
    const float* colscale;         // [G][N] power-of-two scale of B'
    void* j;                       // j[cell * ldj + g * N + n]
    long long ldj;
    int j_f64;
    long long wait_polls;          // polls before a wait on another role gives up (kStatTimeout)
    int* status;
};

size_t emis_tc_smem_bytes();
// ntile: the tile's wavelength columns, 256 or 128 (p.ntiles = ceil(N / ntile); the B maps'
// boxes are ntile rows high)
cudaError_t launch_emis_tc(const EmisTcParams& p, bool tf32, bool split, int ntile, int sms, cudaStream_t st);
cudaError_t launch_pack_p(int cells, int G, const int* bin_off, const double* P, long long ldP, const long long* aoff,
                          const int* kp, int split, int tf32, void* A, float* rowscale, cudaStream_t st);
cudaError_t launch_pack_k(int N, int G, const int* bin_off, const double* K, const long long* boff, const int* kp,
                          int split, int tf32, void* B, float* colscale, cudaStream_t st);

}  // namespace heat
