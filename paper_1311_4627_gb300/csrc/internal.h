// Launchers shared between the host API and the kernel translation units.
#pragma once
#include <cuda_runtime.h>

namespace heat {

constexpr int kGLPoints = 16;

struct PatF64;
struct PatF32;
struct SoftF64;
struct RowEnt32;

// ---- grain set-up (k_setup.cu)
cudaError_t set_gauss_legendre(const double* x, const double* w);
cudaError_t launch_cooling(int N, const double* lam, const double* cabs, const int* bin_off, int G, const double* T,
                           const double* E, double* Cf, const int2* work, int n_work, cudaStream_t st);
cudaError_t launch_kexp(int N, int nbt, const double* K, int* kexp, cudaStream_t st);
cudaError_t launch_planck(int N, int nbt, const double* lam, const double* cabs, const int* bin_grain, const double* T,
                          const double* E, const double* w, double* K, double* Kw, cudaStream_t st);

// ---- per-solve kernels (k_build.cu: field, build; k_recur.cu: recursion)

// Per-grain device tables consumed by the solve kernels.
struct GrainDev {
    int N;              // wavelengths
    int G;              // grains
    int nbt;            // total bins over grains
    const double* lam;  // [N]
    const double* dln;  // [N-1] ln(lambda_{n+1}/lambda_n)
    const int* bin_off; // [G+1]
    const double* Cact;     // [G][N] C_n if the C segment n is active (both ends > 0), else 0
    const double* sC;       // [G][N] log-log slope of C on segment n (0 if inactive)
    const float* lam32;     // [N]   FP32 copies for the FP32 build
    const float* dln32;     // [N-1]
    const float* ca32;      // [G][N] C_n lambda_n^2 / h on active C segments, else 0
    const float* ce32;      // [G][N] c C_n lambda_n on active C segments, else 0
    const float* sC32;      // [G][N]
    const float* invdE32;   // [nbt]
    const double* invC;     // [nbt] 1/T_{f-1,f} (0 where the cooling rate is 0 and for f = 0)
    const double* cde;      // [nbt] T_{f-1,f} (E_f - E_{f-1}) (0 for f = 0): emitted power of bin f
    const double* E;        // [nbt] bin enthalpies
    const double* invdE;    // [nbt] 1/(E_{j+1}-E_j) (0 for the last bin)
    const int* rowptr;      // [nbt + G] per grain, rows f = 0..M: band elements of row f at
                            //   rowptr[off_g + g + f] .. rowptr[off_g + g + f + 1] (global indices)
    const int* wmax;        // [G] widest band row of grain g (selects the recursion's window size)
    long long band_total;   // band elements of all grains (per cell)
    int max_bins;           // largest bins per grain
    int band_max;           // largest band (elements per cell) of one grain
    int wmax_all;           // widest band row over the grains
    int pat_prefetch;       // nonzero: the FP32 build prefetches into L1 the pattern entry 32 past each segment
    const int* seg_ptr;     // [G][N+1] pattern entries of grain g in segment n at
                            //   seg_ptr[g*(N+1)+n] .. seg_ptr[g*(N+1)+n+1]
    const PatF64* pat64;    // pattern entries (FP64 build)
    const PatF32* pat32;    // pattern entries (FP32 build), then 64 zero entries (prefetch margin)
    const SoftF64* soft;    // [nbt - G] per grain, sorted by segment (descending)
    const int* soft_off;    // [G+1] start of each grain's soft list
    const PointEnt* pent;   // point-rule entries, column by column (u descending within a column)
    const int* pcol;        // [nbt + 1] entries of column j of grain g at pcol[off_g + j] .. pcol[off_g + j + 1]
    const int* kexp;        // [nbt] biased binary exponent of max_lambda K[i][lambda] (-100000: none)
    const RowEnt32* rent;   // [band_total] every band element in band (row) order, for the fused kernel
};

// Per-chunk scratch.
struct ChunkDev {
    int cells;          // valid cells in the chunk
    int Cc;             // padded cells (multiple of 32)
    int NG;             // Cc / 32 cell groups
    const int2* tasks;  // [G * NG] (grain, group), largest work first (recursion order)
    const int2* btasks; // the same pairs in the build's order, or null (then `tasks`)
    int n_tasks;
    // field tables, transposed [N][Cc]
    double* ua64; double* su64;
    float* ua32; float* su32;  // FP32 build: su32 unused; ua32 holds float2 (u_n, su_n) pairs
    // band of B, [NG][band_total][32]: element e of group grp, lane l at (grp*band_total + e)*32 + l
    double* Bb64;
    float* Bb32;
    // per-group bin arrays [NG][nbt][32]
    double* xs;         // X history of the recursion
    unsigned short* ep; // rescale epoch at which each stored X was last written
    double* pabs;       // [Cc][G] absorbed power c int Omega dlambda (erg/s)
    double* P;          // [Cc][nbt] output distributions (row stride ldP)
    long long ldP;
    double* ledger;     // [cells][G][2] energy check (absorbed, emitted), or null
    int* status;
    int small;          // 1: the solve has few cells (kSmallCells): element-parallel kernels
    int point;          // 1: point-rule heating (HEAT_HEATING_POINT, FP64 build only)
    int prune;          // L > 0: stop a spectrum's recursion at the tail test with threshold 2^-L; 0: off
    int* work;          // [2] task counters of the persistent launches (the recursion uses [1]), zero
                        //   before the launches; null: one warp per task
    float* phs;         // fused kernel: per resident warp, the photon prefix table [N+1][32] (FP32,
                        //   sign bit = the segment's short-series flag); null otherwise
    int blocks_per_sm;  // cap on the persistent recursion's resident blocks per SM (0: occupancy)
    // The tensor-core emissivity's P operand, written by k_recur's epilogue (null: k_pack_p
    // packs P afterwards, and P is always written).  Per grain, A'_g [cells][Kp_g] at packA +
    // pack_aoff[g] elements (2 bytes, BF16, or 4, TF32), [P_hi | P_lo] when split, and the
    // row scales [cells][G].  With packA set, P may be null (P not requested).
    void* packA;
    const long long* pack_aoff;
    const int* pack_kp;
    float* pack_rowscale;
    int pack_tf32, pack_split;
};

// Solves of at most this many cells use the element-parallel build and recursion (a block
// per (cell, grain) for the build, a warp per spectrum with lanes over the band for the
// recursion) instead of lane = cell, which would leave most lanes idle.  The choice is
// made on the whole solve's cell count, so chunking never changes it.
constexpr int kSmallCells = 16;

cudaError_t launch_field(const GrainDev& g, const void* u, int dtype, long long cell0, const ChunkDev& ch, int build,
                         cudaStream_t st);
cudaError_t launch_build(const GrainDev& g, const ChunkDev& ch, int build, cudaStream_t st);
cudaError_t launch_recur(const GrainDev& g, const ChunkDev& ch, int build, cudaStream_t st);
// The mixed path (FP32 build, integral heating, more than kSmallCells cells) with the matrix
// build fused into the persistent recursion (k_fused.cu): B never goes to memory.  Needs
// ch.work and ch.phs sized for fused_warps() warps.
int fused_warps(int n_tasks);  // resident warps of the persistent launch for n_tasks tasks
cudaError_t launch_fused(const GrainDev& g, const ChunkDev& ch, cudaStream_t st);

// ---- thermal-discrete cooling (k_discrete.cu)
// Downward rates of every grain, D_g [nb_g][nb_g] (row l, column u) at D + doff[g]; windows
// of grain g numbered from woff[g] (u(u-1)/2 + l); glx/glw: Gauss-Legendre nodes, weights.
cudaError_t launch_cooling_window(int N, const double* lam, const double* cabs, const int* bin_off, int G,
                                  const double* T, const double* E, const long long* woff, long long n_windows,
                                  const long long* doff, double* D, const double* glx, const double* glw,
                                  cudaStream_t st);
// P (and the ledger) of the chunk's cells x grains by the full stationary solve, `batch`
// spectra at a time, each with an nb x nb rate matrix at q + k * qstride.
// State reduction: states removed per panel, threads per spectrum, and the largest grain whose
// rate matrix is kept in shared memory (row stride nb + 1; 218,880 B at 160 bins).
constexpr int kGthB = 8;
constexpr int kGthThreads = 256;
constexpr int kGthSmemBins = 160;
size_t gth_smem_bytes(int max_bins);
size_t td_fill_smem_bytes(int N);
// Shared memory per block of the few-cell recursion up to which the band is staged there.
constexpr size_t kSmallRecurStage = 100 * 1024;
constexpr int kDiscreteMaxBins = 2048;                // the state reduction's vectors in shared memory
constexpr size_t kMaxSmemPerBlock = 227 * 1024;       // opt-in dynamic shared memory per block
// Spectra are solved in launches of `batch` (rate matrices at q + k * qstride): the k-th
// spectrum from s0 is grain gorder[(s0 + k) / cells], cell (s0 + k) % cells.
long long discrete_batch_spectra(const GrainDev& g, const ChunkDev& ch, long long s0, long long batch);
cudaError_t launch_discrete_fill(const GrainDev& g, const ChunkDev& ch, const double* D, const long long* doff,
                                 const int* gorder, double* q, long long qstride, long long s0, long long n,
                                 cudaStream_t st);
cudaError_t launch_discrete_gth(const GrainDev& g, const ChunkDev& ch, const int* gorder, double* q, long long qstride,
                                long long s0, long long n, cudaStream_t st);

// ---- emissivity (k_emis.cu)
// C[z][m][n] = sum_{k in [koff[z], koff[z+1])} A[m][k] B[k][n] for z < nz, m < M, n < N;
// koff is a device array of nz+1 offsets; C[z] starts at C + z * zstride_c.
cudaError_t launch_gemm_f64(int M, int N, int nz, const int* koff, const double* A, long long lda,
                            const double* B, long long ldb, void* C, long long ldc, long long zstride_c, int c_is_f32,
                            cudaStream_t st);

}  // namespace heat
