// Per-solve kernels: field tables, the matrix build (B band, intra-bin terms) and the
// Guhathakurta-Draine recursion (Eq. bmatrix, Eq. xf, Eq. renormalization).
//
// Work unit ("task") = one grain x 32 cells; one warp per task, one lane per cell.
// All lanes of a warp walk the same band of the same grain, so neither kernel has
// divergence or cross-lane reductions: in the recursion each band element costs one
// FP64 FMA per cell.
#include "common.cuh"
#include "internal.h"

namespace heat {

// ---------------------------------------------------------------------------
// k_field: transpose the chunk's fields to [N][Cc] and form the log-log slope of
// u on each segment.  ua_n = u_n where both ends of segment n are > 0 (else 0),
// su_n = ln(u_{n+1}/u_n) / ln(lambda_{n+1}/lambda_n) (else 0); ua, su = 0 at n = N-1
// and for padding cells.  Negative or non-finite input sets kStatBadInput.
// Block (32, 8) handles 32 wavelengths x 32 cells.
template <typename TU, typename TO>
__global__ void k_field(int N, const double* __restrict__ dln, const TU* __restrict__ u, long long cell0, int cells,
                        int Cc, TO* __restrict__ ua, TO* __restrict__ su, int* status) {
    __shared__ TO t_ua[32][33];
    __shared__ TO t_su[32][33];
    int n0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    int tx = threadIdx.x, ty = threadIdx.y;
    int bad = 0;
    for (int k = 0; k < 4; ++k) {
        int c = c0 + ty + 8 * k, n = n0 + tx;
        TO a = 0, s = 0;
        if (c < cells && n < N) {
            const TU* row = u + (size_t)(cell0 + c) * N;
            double un = (double)row[n];
            if (!(un >= 0.0 && un < INFINITY)) bad = 1;
            if (n < N - 1) {
                double un1 = (double)row[n + 1];
                if (sizeof(TO) == 8) {
                    if (un > 0.0 && un1 > 0.0 && un1 < INFINITY && un < INFINITY) {
                        a = (TO)un;
                        s = (TO)(log(un1 / un) / dln[n]);
                    }
                } else {
                    float fa = (float)un, fb = (float)un1;
                    if (fa > 0.0f && fb > 0.0f && fa < INFINITY && fb < INFINITY) {
                        a = (TO)fa;
                        s = (TO)(logf(fb / fa) / (float)dln[n]);
                    }
                }
            }
        }
        t_ua[ty + 8 * k][tx] = a;
        t_su[ty + 8 * k][tx] = s;
    }
    __syncthreads();
    for (int k = 0; k < 4; ++k) {
        int n = n0 + ty + 8 * k, c = c0 + tx;
        if (n < N && c < Cc) {
            if (sizeof(TO) == 8) {
                ua[(size_t)n * Cc + c] = t_ua[tx][ty + 8 * k];
                su[(size_t)n * Cc + c] = t_su[tx][ty + 8 * k];
            } else {  // FP32 build: interleaved (u, slope) pairs, one 8-byte load per element
                float2 v = make_float2((float)t_ua[tx][ty + 8 * k], (float)t_su[tx][ty + 8 * k]);
                ((float2*)ua)[(size_t)n * Cc + c] = v;
            }
        }
    }
    if (bad) atomicOr(status, kStatBadInput);
}

// ---------------------------------------------------------------------------
// k_build: the matrix-build kernel.  One warp per task (grain x 32 cells), one lane
// per cell.  With Omega = u C on the log-log interpolant (Eq. interpolation), slope
// s_n and q = s_n + p + 1 on segment n:
//   segment integral   int Omega lambda^p = Omega_n lambda_n^{p+1} dln_n E1(q dln_n)
//   photon prefix      Phi_n = (1/h) sum_{m<n} int_m Omega lambda       (cumulative sum: FP64 in
//                      the FP64 build, compensated FP32 in the FP32 build)
//   band element       B_fj = Phi(lambda_fj) = Phi_n + (Omega_n lambda_n^2/h) t E1(q t)
//                      (Eq. bmatrix telescoped: the bins' wavelength ranges tile [0, lambda_fj])
//   intra-bin term     W_j = c int_{hc/(Elo_{j+1}-E_j)}^{lambda_{N-1}} Omega, added to the diagonal
//                      element: B_{j+1,j} += W_j/(E_{j+1}-E_j)
//   absorbed power     c int Omega over the grid
// The segments are walked in order; every band element whose transition wavelength
// falls in the current segment (the grain's pattern list) is written to the band
// storage Bb, so the recursion streams B instead of gathering tables.
template <int BUILD>
__device__ __forceinline__ void build_task(const GrainDev& gd, const ChunkDev& ch, int task, int lane) {
    const int N = gd.N, Cc = ch.Cc;
    const int2 tk = (ch.btasks ? ch.btasks : ch.tasks)[task];
    int g = tk.x, grp = tk.y;
    int off = gd.bin_off[g];
    int cc = grp * 32 + lane;
    size_t bb = (size_t)grp * gd.band_total * 32 + lane;  // + e * 32
    const int* sp = gd.seg_ptr + (size_t)g * (N + 1);
    const SoftF64* soft = gd.soft;
    int p = gd.soft_off[g], p1 = gd.soft_off[g + 1];
    double Phi = 0.0;

    if (BUILD == 0) {
        const double* Cact = gd.Cact + (size_t)g * N;
        const double* sC = gd.sC + (size_t)g * N;
        for (int n = 0; n < N - 1; ++n) {
            double ua = ch.ua64[(size_t)n * Cc + cc], su = ch.su64[(size_t)n * Cc + cc];
            double om = ua * Cact[n];
            double q1 = su + sC[n] + 2.0;
            double ln = gd.lam[n];
            double a = om * ln * ln / kH;
            double aq = (q1 != 0.0) ? a / q1 : a;
            for (int k = sp[n]; k < sp[n + 1]; ++k) {
                PatF64 pt = gd.pat64[k];
                double B = Phi + (q1 != 0.0 ? aq * expm1(q1 * pt.t) : aq * pt.t);
                ch.Bb64[bb + (size_t)pt.e * 32] = B;
            }
            if (om > 0.0) Phi += a * gd.dln[n] * e1d(q1 * gd.dln[n]);
        }
        for (int k = sp[N - 1]; k < sp[N]; ++k) ch.Bb64[bb + (size_t)gd.pat64[k].e * 32] = Phi;

        // intra-bin terms go into the diagonal elements (j+1, j) of the band
        auto put64 = [&](const SoftF64& sf, double v) {
            size_t ix = bb + (size_t)sf.e_diag * 32;
            ch.Bb64[ix] = (sf.diag_in_band ? ch.Bb64[ix] : 0.0) + v;
        };
        while (p < p1 && soft[p].n == N - 1) {
            put64(soft[p], 0.0);
            ++p;
        }
        double Psi = 0.0;  // int Omega from lambda_{n+1} to lambda_{N-1}
        for (int n = N - 2; n >= 0; --n) {
            double ua = ch.ua64[(size_t)n * Cc + cc], su = ch.su64[(size_t)n * Cc + cc];
            double om = ua * Cact[n];
            double q0 = su + sC[n] + 1.0;
            double b = om * gd.lam[n];
            double dl = gd.dln[n];
            while (p < p1 && soft[p].n == n) {
                SoftF64 sf = soft[p];
                double part = 0.0;
                if (om > 0.0) {
                    double L = dl - sf.t;
                    part = b * exp(q0 * sf.t) * L * e1d(q0 * L);
                }
                put64(sf, kC * (part + Psi) * gd.invdE[off + sf.j]);
                ++p;
            }
            if (om > 0.0) Psi += b * dl * e1d(q0 * dl);
        }
        for (; p < p1; ++p) put64(soft[p], kC * Psi * gd.invdE[off + soft[p].j]);
        if (ch.pabs) ch.pabs[(size_t)cc * gd.G + g] = kC * Psi;
    } else {
        const float* ca = gd.ca32 + (size_t)g * N;
        const float* ce = gd.ce32 + (size_t)g * N;
        const float* sC = gd.sC32 + (size_t)g * N;
        const float2* uasu = (const float2*)ch.ua32;
        float* Bb = ch.Bb32 + bb;
        float2 us_next = uasu[cc];
        Sum32 Phi32;  // the photon prefix, compensated in FP32
        for (int n = 0; n < N - 1; ++n) {
            float2 us = us_next;
            if (n + 1 < N - 1) us_next = uasu[(size_t)(n + 1) * Cc + cc];  // one segment ahead
            float ua = us.x, su = us.y;
            float phi = Phi32.val();
            int k = sp[n], k1 = sp[n + 1];
            // every element's argument is z = q t with t in [0, dln]: when |q| dln <= 1/4 the
            // short series serves the whole segment.  The test is per lane (per cell), so a
            // cell's values do not depend on the cells sharing its warp; lanes normally agree
            if (short_series(su, sC[n], gd.dln32[n])) {
                for (; k + 2 <= k1; k += 2) {
                    PatF32 a0 = gd.pat32[k], a1 = gd.pat32[k + 1];
                    __stcs(Bb + (size_t)a0.e * 32, fmaf(ua * a0.cat, e1f_small(fmaf(su, a0.t, a0.zt)), phi));
                    __stcs(Bb + (size_t)a1.e * 32, fmaf(ua * a1.cat, e1f_small(fmaf(su, a1.t, a1.zt)), phi));
                }
                if (k < k1) {
                    PatF32 a0 = gd.pat32[k];
                    __stcs(Bb + (size_t)a0.e * 32, fmaf(ua * a0.cat, e1f_small(fmaf(su, a0.t, a0.zt)), phi));
                }
            } else {
                for (; k + 2 <= k1; k += 2) {
                    PatF32 a0 = gd.pat32[k], a1 = gd.pat32[k + 1];
                    __stcs(Bb + (size_t)a0.e * 32, fmaf(ua * a0.cat, e1f(fmaf(su, a0.t, a0.zt)), phi));
                    __stcs(Bb + (size_t)a1.e * 32, fmaf(ua * a1.cat, e1f(fmaf(su, a1.t, a1.zt)), phi));
                }
                if (k < k1) {
                    PatF32 a0 = gd.pat32[k];
                    __stcs(Bb + (size_t)a0.e * 32, fmaf(ua * a0.cat, e1f(fmaf(su, a0.t, a0.zt)), phi));
                }
            }
            float a = ua * ca[n];
            if (a > 0.0f) {
                float dl = gd.dln32[n];
                Phi32.add(a * dl * e1f((su + sC[n] + 2.0f) * dl));
            }
        }
        float phi_end = Phi32.val();
        for (int k = sp[N - 1]; k < sp[N]; ++k) Bb[gd.pat32[k].e * 32] = phi_end;

        auto put32 = [&](const SoftF64& sf, float v) {
            float* q = Bb + (size_t)sf.e_diag * 32;
            *q = (sf.diag_in_band ? *q : 0.0f) + v;
        };
        while (p < p1 && soft[p].n == N - 1) {
            put32(soft[p], 0.0f);
            ++p;
        }
        Sum32 Psi32;  // c int Omega from lambda_{n+1} to lambda_{N-1} (compensated FP32 sum)
        us_next = uasu[(size_t)(N - 2) * Cc + cc];
        for (int n = N - 2; n >= 0; --n) {
            float2 us = us_next;
            if (n > 0) us_next = uasu[(size_t)(n - 1) * Cc + cc];
            float ua = us.x, su = us.y;
            float b = ua * ce[n];
            float q0 = su + sC[n] + 1.0f;
            float dl = gd.dln32[n];
            while (p < p1 && soft[p].n == n) {
                SoftF64 sf = soft[p];
                float part = 0.0f;
                if (b > 0.0f) {
                    float ts = (float)sf.t;
                    float L = dl - ts;
                    part = b * __expf(q0 * ts) * L * e1f(q0 * L);
                }
                put32(sf, (part + Psi32.val()) * gd.invdE32[off + sf.j]);
                ++p;
            }
            if (b > 0.0f) Psi32.add(b * dl * e1f(q0 * dl));
        }
        float psi_end = Psi32.val();
        for (; p < p1; ++p) put32(soft[p], psi_end * gd.invdE32[off + soft[p].j]);
        if (ch.pabs) ch.pabs[(size_t)cc * gd.G + g] = Psi32.wide();
    }
}

// Task loop of the persistent launches: with ch.work set, each warp takes the next task of
// the list from an atomic counter (dynamic scheduling per warp, in the list's order, as the
// paper's dynamic OpenMP schedule does per thread); without it, one warp per task.
template <typename F>
__device__ __forceinline__ void for_each_task(const ChunkDev& ch, int counter, F&& run) {
    const int lane = threadIdx.x & 31;
    if (!ch.work) {
        const int task = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        if (task < ch.n_tasks) run(task, lane);
        return;
    }
    for (;;) {
        int task = 0;
        if (lane == 0) task = atomicAdd(ch.work + counter, 1);
        task = __shfl_sync(0xffffffffu, task, 0);
        if (task >= ch.n_tasks) return;
        run(task, lane);
    }
}

template <int BUILD>
__global__ void __launch_bounds__(128) k_build(GrainDev gd, ChunkDev ch) {
    for_each_task(ch, 0, [&](int task, int lane) { build_task<BUILD>(gd, ch, task, lane); });
}

// ---------------------------------------------------------------------------
// k_recur: the recursion kernel.  X_0 = 1,
//   X_f = (sum_{j in band(f)} B_fj X_j) / T_{f-1,f}                              (Eq. xf)
// in FP64, where the band holds every j whose transition wavelength lies on the grid
// (all other B_fj are exactly zero) plus the diagonal j = f-1, which also carries the
// intra-bin term; then P = X / sum X (Eq. renormalization) is written to P[cell][off_g + i].
// Overflow guard: when X_f >= 2^800 every X is to be multiplied by 2^-800 (exact).  Only
// the values later rows still read (j >= the next row's band start), the register window
// and the running sum are scaled at once; each stored X keeps the epoch (count of
// rescales) it was last written in, and the normalisation applies the missing powers of
// two, so the work is O(band) per rescale instead of O(f) and the result is the same.
// B streams from the band storage in element order with evict-first loads (it is read
// once), eight elements per step, so that the X history stays in L2.
template <int BUILD>
__device__ __forceinline__ double band_b(const float* B32, const double* B64, int e) {
    if (BUILD) return widen_pos(__ldcs(B32 + (size_t)e * 32));
    return __ldcs(B64 + (size_t)e * 32);
}

// B in its stored type (kept in registers ahead of use), and its FP64 value
template <int BUILD>
struct BandRaw {
    using T = double;
    static __device__ __forceinline__ T load(const float*, const double* B64, int e) {
        return __ldcs(B64 + (size_t)e * 32);
    }
    static __device__ __forceinline__ double wide(T v) { return v; }
};
template <>
struct BandRaw<1> {
    using T = float;
    static __device__ __forceinline__ T load(const float* B32, const double*, int e) {
        return __ldcs(B32 + (size_t)e * 32);
    }
    static __device__ __forceinline__ double wide(T v) { return widen_pos(v); }
};

// Window part of a row: element e1-1-k multiplies X_{f-1-k} = w[k] for k < nreg (<= W),
// accumulated into S in element order; a jump into the unrolled tail, so no predicated-off
// FMA occupies the FP64 pipe.
template <int BUILD, int W>
__device__ __forceinline__ void window_tail(int nreg, const typename BandRaw<BUILD>::T (&br)[W],
                                            const double (&w)[W], double& S) {
    using Raw = BandRaw<BUILD>;
    switch (nreg) {
        case 8: if constexpr (W > 7) S = fma(Raw::wide(br[7 % W]), w[7 % W], S);  // fallthrough
        case 7: if constexpr (W > 6) S = fma(Raw::wide(br[6 % W]), w[6 % W], S);  // fallthrough
        case 6: if constexpr (W > 5) S = fma(Raw::wide(br[5 % W]), w[5 % W], S);  // fallthrough
        case 5: if constexpr (W > 4) S = fma(Raw::wide(br[4 % W]), w[4 % W], S);  // fallthrough
        case 4: if constexpr (W > 3) S = fma(Raw::wide(br[3 % W]), w[3 % W], S);  // fallthrough
        case 3: if constexpr (W > 2) S = fma(Raw::wide(br[2 % W]), w[2 % W], S);  // fallthrough
        case 2: if constexpr (W > 1) S = fma(Raw::wide(br[1 % W]), w[1 % W], S);  // fallthrough
        case 1: S = fma(Raw::wide(br[0]), w[0], S);                               // fallthrough
        default: break;
    }
}

// One task: the recursion of grain g for the 32 cells of group grp (lane = cell).  W is
// the register window: the last W values of X, and the window part of each row's band
// (its last min(width, W) elements), prefetched one row ahead.  The row loop's fixed
// cost grows with W, so grains whose rows are all narrow (the large grains: nearly a
// chain) use a small W.
//
// PRUNE (heat_opts.prune_eps > 0, threshold 2^-L): a row f is "small" for a cell when both
// X_f < 2^-L max_{i<=f} X_i and X_f Kmax_f < 2^-L max_{i<=f} X_i Kmax_i (Kmax_i: the bin's
// largest emission kernel over the grid), tested on binary exponents.  Once every row of
// the band window [f - width_f, f] is small, the cell's X_f' for f' > f are set to zero:
// X_f' is a combination of the window's values only, so beyond this point the spectrum
// carries no more than a 2^-L share of the probability or of any wavelength's emission,
// unless it grows again (which a steady state past its mode does not).  The decision is per
// cell, so results do not depend on which cells share a warp; the warp leaves the row loop
// once all its cells have stopped.
template <int BUILD, int W, bool PRUNE>
__device__ __forceinline__ void recur_task(const GrainDev& gd, const ChunkDev& ch, int g, int grp, int lane) {
    using Raw = BandRaw<BUILD>;
    const int nbt = gd.nbt;
    const int off = gd.bin_off[g];
    const int M = gd.bin_off[g + 1] - off - 1;
    const int cc = grp * 32 + lane;
    const size_t xb = ((size_t)grp * nbt + off) * 32 + lane;
    const int* rp = gd.rowptr + off + g;
    const double* ic_row = gd.invC + off;
    double* xl = ch.xs + xb;
    const size_t bb = (size_t)grp * gd.band_total * 32 + lane;
    const float* __restrict__ B32 = ch.Bb32 + (BUILD ? bb : 0);
    const double* __restrict__ B64 = ch.Bb64 + (BUILD ? 0 : bb);
    bool numeric_bad = false;

    unsigned short* epl = ch.ep + xb;
    int epoch = 0;
    xl[0] = 1.0;
    epl[0] = 0;
    double total = 1.0;  // running sum of X, rescaled with it
    // register window: w[k] = X_{f-1-k}; the band's last elements read it instead of
    // reloading what this thread just stored
    double w[W];
#pragma unroll
    for (int k = 0; k < W; ++k) w[k] = 0.0;
    w[0] = 1.0;
    // row pipeline: the band bounds, the cooling rate and the window-part B values of row
    // f+1 are loaded while row f is computed
    int e = rp[1];                       // band of row f: elements [e, e1)
    int e1 = rp[2];
    int e2 = M >= 2 ? rp[3] : e1;        // end of row f+1's band
    double ic = ic_row[1];
    typename Raw::T br[W];               // window part of row f: br[k] = B at element e1-1-k
    {
        const int nr = min(e1 - e, W);
#pragma unroll
        for (int k = 0; k < W; ++k) br[k] = (k < nr) ? Raw::load(B32, B64, e1 - 1 - k) : 0;
    }
    const int e_end = rp[M + 1];
    // L2 prefetch of the B stream, kept 64..96 elements ahead: lane k fetches the
    // 128-byte line of element pf + k (lines of all 32 lanes of one element)
    const size_t lane_base = bb - lane;
    int pf = e;
    // tail pruning state: running maxima of the true binary exponents (epoch included) of X
    // and of X Kmax, the last row that was not small, whether this cell has stopped
    const int* kx = gd.kexp + off;
    int xmax = 1023, cmax = 0, last_big = 0, f_last = M;
    bool stopped = false;
    if constexpr (PRUNE) cmax = 1023 + kx[0];
    for (int f = 1; f <= M; ++f) {
        int kf = 0;
        if constexpr (PRUNE) kf = kx[f];
        // next row's loads
        const bool more = f < M;
        const int e3 = f + 2 <= M ? rp[f + 3] : e2;
        const double ic_n = more ? ic_row[f + 1] : 0.0;
        const int nr_n = more ? min(e2 - e1, W) : 0;
        typename Raw::T br_n[W];
#pragma unroll
        for (int k = 0; k < W; ++k) br_n[k] = (k < nr_n) ? Raw::load(B32, B64, e2 - 1 - k) : 0;
        while (pf < e1 + 64 && pf < e_end) {
            int q = pf + lane;
            if (q < e_end) {
                const void* a = BUILD ? (const void*)(ch.Bb32 + lane_base + (size_t)q * 32)
                                      : (const void*)(ch.Bb64 + lane_base + (size_t)q * 32);
                asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
            }
            pf += 32;
        }
        const int width = e1 - e;          // band of row f: j in [f - width, f)
        const int nreg = min(width, W);    // its last nreg elements come from the window
        const int e_mem = e1 - nreg;       // elements before e_mem read X from memory
        // one accumulator, in element order: the SM sub-partition's FP64 unit, shared by the
        // warps on it, is the bound, not this warp's dependent FMA chain
        double S = 0.0;
        if (e < e_mem) {
            int j = f - width;
            // batches of 8 elements, two register sets: the loads of the next batch are in
            // flight while this batch's FMAs run (no register copy waits on a load)
            const int nb = (e_mem - e) >> 3;
            if (nb > 0) {
                typename Raw::T bA[8], bB[8];
                double xA[8], xB[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) bA[k] = Raw::load(B32, B64, e + k);
#pragma unroll
                for (int k = 0; k < 8; ++k) xA[k] = xl[(j + k) * 32];
                int i = 0;
                for (; i + 2 <= nb; i += 2) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) bB[k] = Raw::load(B32, B64, e + 8 + k);
#pragma unroll
                    for (int k = 0; k < 8; ++k) xB[k] = xl[(j + 8 + k) * 32];
#pragma unroll
                    for (int k = 0; k < 8; ++k) S = fma(Raw::wide(bA[k]), xA[k], S);
                    if (i + 2 < nb) {
#pragma unroll
                        for (int k = 0; k < 8; ++k) bA[k] = Raw::load(B32, B64, e + 16 + k);
#pragma unroll
                        for (int k = 0; k < 8; ++k) xA[k] = xl[(j + 16 + k) * 32];
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) S = fma(Raw::wide(bB[k]), xB[k], S);
                    e += 16;
                    j += 16;
                }
                if (i < nb) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) S = fma(Raw::wide(bA[k]), xA[k], S);
                    e += 8;
                    j += 8;
                }
            }
            for (; e < e_mem; ++e, ++j) S = fma(band_b<BUILD>(B32, B64, e), xl[j * 32], S);
        }
        window_tail<BUILD, W>(nreg, br, w, S);
        double X = S * ic;
        if (__double2hiint(ic) == 0 && __double2loint(ic) == 0) {  // zero cooling rate
            X = 0.0;
            if (S != 0.0 && !(PRUNE && stopped)) numeric_bad = true;
        }
        if constexpr (PRUNE) {
            if (stopped) {
                X = 0.0;
            } else {
                const int L = ch.prune;
                const int xe = ((__double2hiint(X) >> 20) & 0x7ff) + 800 * epoch;
                const int ce = xe + kf;
                xmax = max(xmax, xe);
                cmax = max(cmax, ce);
                if (!(xe < xmax - L && ce < cmax - L)) last_big = f;
                stopped = last_big < f - width;
            }
        }
        xl[f * 32] = X;
        epl[f * 32] = (unsigned short)epoch;
        total += X;
#pragma unroll
        for (int k = W - 1; k > 0; --k) w[k] = w[k - 1];
        w[0] = X;
        if (above_rescale(X)) {
            ++epoch;
            const int lo = more ? (f + 1) - (e2 - e1) : f + 1;  // next row's band start
            for (int i = lo; i <= f; ++i) {
                xl[i * 32] *= kRescaleSmall;
                epl[i * 32] = (unsigned short)epoch;
            }
            total *= kRescaleSmall;
#pragma unroll
            for (int k = 0; k < W; ++k) w[k] *= kRescaleSmall;
        }
        if constexpr (PRUNE) {
            if (__all_sync(0xffffffffu, stopped)) {
                f_last = f;
                break;
            }
        }
        // rotate the row pipeline
        e = e1;
        e1 = e2;
        e2 = e3;
        ic = ic_n;
#pragma unroll
        for (int k = 0; k < W; ++k) br[k] = br_n[k];
    }
    if (cc < ch.cells) {
        const double inv = 1.0 / total;
        double* prow = ch.P + (size_t)cc * ch.ldP + off;
        double emit = 0.0;
        const double* cde = gd.cde + off;
        const int i_end = PRUNE ? f_last : M;
        for (int i = 0; i <= i_end; ++i) {
            const int d = epoch - (int)epl[i * 32];  // rescales this value has not seen
            const double x = xl[i * 32];
            // scale X first (as the plain rescale would have), then normalise: the factor
            // alone could underflow where the product is still a normal number
            const double p = d == 0 ? x * inv : ldexp(x, -800 * d) * inv;
            prow[i] = p;
            if (ch.ledger) emit = fma(p, cde[i], emit);
        }
        if constexpr (PRUNE)
            for (int i = f_last + 1; i <= M; ++i) prow[i] = 0.0;  // rows past a pruned tail
        if (ch.ledger) {
            double* lg = ch.ledger + ((size_t)cc * gd.G + g) * 2;
            lg[0] = ch.pabs[(size_t)cc * gd.G + g];
            lg[1] = emit;
        }
    }
    if (numeric_bad) atomicOr(ch.status, kStatNumeric);
}

template <int BUILD, bool PRUNE>
__global__ void __launch_bounds__(128, 4) k_recur(GrainDev gd, ChunkDev ch) {
    for_each_task(ch, 1, [&](int task, int lane) {
        const int g = ch.tasks[task].x, grp = ch.tasks[task].y;
        const int wm = gd.wmax[g];  // warp-uniform
        if (wm <= 1)
            recur_task<BUILD, 1, PRUNE>(gd, ch, g, grp, lane);
        else if (wm <= 2)
            recur_task<BUILD, 2, PRUNE>(gd, ch, g, grp, lane);
        else if (wm <= 4)
            recur_task<BUILD, 4, PRUNE>(gd, ch, g, grp, lane);
        else
            recur_task<BUILD, 8, PRUNE>(gd, ch, g, grp, lane);
    });
}

// ---------------------------------------------------------------------------
// Element-parallel kernels for solves of few cells (ChunkDev::small).  They compute the same
// quantities as k_build / k_recur with the same expressions; the build's cumulative sums
// run in the same order (one thread), so B is bit-identical; the recursion sums each row
// across lanes, so its rounding differs from the lane-per-cell kernel's.

// Per-segment pieces of the build, shared in form with k_build (same operations, same order).
struct SegF64 {
    double om, q1, q0, dl, a;
};
__device__ __forceinline__ SegF64 seg64(const GrainDev& gd, int g, int n, double ua, double su) {
    SegF64 r;
    r.om = ua * gd.Cact[(size_t)g * gd.N + n];
    const double sc = gd.sC[(size_t)g * gd.N + n];
    r.q1 = su + sc + 2.0;
    r.q0 = su + sc + 1.0;
    const double ln = gd.lam[n];
    r.a = r.om * ln * ln / kH;
    r.dl = gd.dln[n];
    return r;
}

// Block per (cell, grain): 256 threads, dynamic shared memory 2 N doubles.
template <int BUILD>
__global__ void __launch_bounds__(256) k_build_small(GrainDev gd, ChunkDev ch) {
    extern __shared__ double sm[];
    double* sPhi = sm;          // [N]: Phi before segment n (exclusive prefix), then Phi at the end
    double* sPsi = sm + gd.N;   // [N]: Psi after the segments above n (exclusive suffix)
    __shared__ double sPhiEnd, sPsiTot;
    __shared__ float sPsiEnd32;  // FP32 build: the FP32 value of the compensated total
    const int N = gd.N, Cc = ch.Cc;
    const int cell = blockIdx.x / gd.G, g = blockIdx.x % gd.G;
    if (cell >= ch.cells) return;
    const int grp = cell >> 5, lc = cell & 31;
    const int off = gd.bin_off[g];
    const size_t bb = (size_t)grp * gd.band_total * 32 + lc;
    const int* sp = gd.seg_ptr + (size_t)g * (N + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float2* uasu = (const float2*)ch.ua32;
    // 1. segment increments, in parallel
    for (int n = tid; n < N - 1; n += blockDim.x) {
        double dphi = 0.0, dpsi = 0.0;
        if (BUILD == 0) {
            const SegF64 s = seg64(gd, g, n, ch.ua64[(size_t)n * Cc + cell], ch.su64[(size_t)n * Cc + cell]);
            if (s.om > 0.0) {
                dphi = s.a * s.dl * e1d(s.q1 * s.dl);
                dpsi = s.om * gd.lam[n] * s.dl * e1d(s.q0 * s.dl);
            }
        } else {
            const float2 us = uasu[(size_t)n * Cc + cell];
            const float ua = us.x, su = us.y;
            const float sc = gd.sC32[(size_t)g * N + n], dl = gd.dln32[n];
            const float a = ua * gd.ca32[(size_t)g * N + n];
            if (a > 0.0f) dphi = widen_pos(a * dl * e1f((su + sc + 2.0f) * dl));
            const float b = ua * gd.ce32[(size_t)g * N + n];
            if (b > 0.0f) dpsi = widen_pos(b * dl * e1f((su + sc + 1.0f) * dl));
        }
        sPhi[n] = dphi;
        sPsi[n] = dpsi;
    }
    __syncthreads();
    // 2. the cumulative sums, in the lane-per-cell kernel's order and arithmetic (FP64 build:
    // FP64 sums; FP32 build: compensated FP32 sums, whose FP32 values are kept)
    if (tid == 0) {
        if (BUILD == 0) {
            double Phi = 0.0;
            for (int n = 0; n < N - 1; ++n) {
                const double d = sPhi[n];
                sPhi[n] = Phi;
                Phi += d;
            }
            sPhiEnd = Phi;
        } else {
            Sum32 Phi;
            for (int n = 0; n < N - 1; ++n) {
                const float d = (float)sPhi[n];
                sPhi[n] = Phi.val();
                Phi.add(d);
            }
            sPhiEnd = Phi.val();
        }
    } else if (tid == 32) {
        if (BUILD == 0) {
            double Psi = 0.0;
            for (int n = N - 2; n >= 0; --n) {
                const double d = sPsi[n];
                sPsi[n] = Psi;
                Psi += d;
            }
            sPsiTot = Psi;
        } else {
            Sum32 Psi;
            for (int n = N - 2; n >= 0; --n) {
                const float d = (float)sPsi[n];
                sPsi[n] = Psi.val();
                Psi.add(d);
            }
            sPsiTot = Psi.wide();
            sPsiEnd32 = Psi.val();
        }
    }
    __syncthreads();
    // 3. band elements: warp per segment, lanes over its pattern entries
    for (int n = warp; n < N - 1; n += blockDim.x >> 5) {
        const int k0 = sp[n], k1 = sp[n + 1];
        if (k0 == k1) continue;
        if (BUILD == 0) {
            const SegF64 s = seg64(gd, g, n, ch.ua64[(size_t)n * Cc + cell], ch.su64[(size_t)n * Cc + cell]);
            const double aq = (s.q1 != 0.0) ? s.a / s.q1 : s.a;
            const double Phi = sPhi[n];
            for (int k = k0 + lane; k < k1; k += 32) {
                const PatF64 pt = gd.pat64[k];
                ch.Bb64[bb + (size_t)pt.e * 32] = Phi + (s.q1 != 0.0 ? aq * expm1(s.q1 * pt.t) : aq * pt.t);
            }
        } else {
            const float2 us = uasu[(size_t)n * Cc + cell];
            const float ua = us.x, su = us.y;
            const float phi = __double2float_rn(sPhi[n]);
            const bool sh = short_series(su, gd.sC32[(size_t)g * N + n], gd.dln32[n]);
            for (int k = k0 + lane; k < k1; k += 32) {
                const PatF32 a0 = gd.pat32[k];
                const float z = fmaf(su, a0.t, a0.zt);
                ch.Bb32[bb + (size_t)a0.e * 32] = fmaf(ua * a0.cat, sh ? e1f_small(z) : e1f(z), phi);
            }
        }
    }
    for (int k = sp[N - 1] + tid; k < sp[N]; k += blockDim.x) {
        if (BUILD == 0)
            ch.Bb64[bb + (size_t)gd.pat64[k].e * 32] = sPhiEnd;
        else
            ch.Bb32[bb + (size_t)gd.pat32[k].e * 32] = __double2float_rn(sPhiEnd);
    }
    __syncthreads();  // the intra-bin terms add to diagonal elements written above
    // 4. intra-bin terms, one per soft entry (each has its own diagonal element)
    for (int p = gd.soft_off[g] + tid; p < gd.soft_off[g + 1]; p += blockDim.x) {
        const SoftF64 sf = gd.soft[p];
        if (BUILD == 0) {
            double v = 0.0;
            if (sf.n == N - 1) {
                v = 0.0;
            } else if (sf.n >= 0) {
                const SegF64 s = seg64(gd, g, sf.n, ch.ua64[(size_t)sf.n * Cc + cell],
                                       ch.su64[(size_t)sf.n * Cc + cell]);
                double part = 0.0;
                if (s.om > 0.0) {
                    const double L = s.dl - sf.t;
                    part = s.om * gd.lam[sf.n] * exp(s.q0 * sf.t) * L * e1d(s.q0 * L);
                }
                v = kC * (part + sPsi[sf.n]) * gd.invdE[off + sf.j];
            } else {
                v = kC * sPsiTot * gd.invdE[off + sf.j];
            }
            const size_t ix = bb + (size_t)sf.e_diag * 32;
            ch.Bb64[ix] = (sf.diag_in_band ? ch.Bb64[ix] : 0.0) + v;
        } else {
            float v = 0.0f;
            if (sf.n == N - 1) {
                v = 0.0f;
            } else if (sf.n >= 0) {
                const float2 us = uasu[(size_t)sf.n * Cc + cell];
                const float b = us.x * gd.ce32[(size_t)g * N + sf.n];
                const float q0 = us.y + gd.sC32[(size_t)g * N + sf.n] + 1.0f;
                const float dl = gd.dln32[sf.n];
                float part = 0.0f;
                if (b > 0.0f) {
                    const float ts = (float)sf.t;
                    const float L = dl - ts;
                    part = b * __expf(q0 * ts) * L * e1f(q0 * L);
                }
                v = (part + __double2float_rn(sPsi[sf.n])) * gd.invdE32[off + sf.j];
            } else {
                v = sPsiEnd32 * gd.invdE32[off + sf.j];
            }
            float* q = ch.Bb32 + bb + (size_t)sf.e_diag * 32;
            *q = (sf.diag_in_band ? *q : 0.0f) + v;
        }
    }
    if (tid == 0 && ch.pabs) ch.pabs[(size_t)cell * gd.G + g] = BUILD == 0 ? kC * sPsiTot : sPsiTot;
}

// Warp per spectrum, lanes over each row's band; X history in shared memory
// (dynamic: max_bins doubles per warp).  Same recursion (Eq. xf), rescale, normalisation and
// tail pruning as k_recur; each row's sum is reduced across lanes.
template <int BUILD, bool PRUNE>
__global__ void __launch_bounds__(128) k_recur_small(GrainDev gd, ChunkDev ch) {
    extern __shared__ double smx[];
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= ch.cells * gd.G) return;
    double* xs = smx + (size_t)(threadIdx.x >> 5) * gd.max_bins;
    const int cell = w / gd.G, g = w % gd.G;
    const int grp = cell >> 5, lc = cell & 31;
    const int off = gd.bin_off[g];
    const int M = gd.bin_off[g + 1] - off - 1;
    const int* rp = gd.rowptr + off + g;
    const double* ic_row = gd.invC + off;
    const size_t bb = (size_t)grp * gd.band_total * 32 + lc;
    const float* B32 = ch.Bb32 + (BUILD ? bb : 0);
    const double* B64 = ch.Bb64 + (BUILD ? 0 : bb);
    bool numeric_bad = false;
    if (lane == 0) xs[0] = 1.0;
    double total = 1.0;
    const int* kx = gd.kexp + off;
    const int L = ch.prune;
    int xmax = 1023, cmax = PRUNE ? 1023 + kx[0] : 0, last_big = 0, f_last = M, shift = 0;
    __syncwarp();
    for (int f = 1; f <= M; ++f) {
        const int e0 = rp[f], width = rp[f + 1] - e0, j0 = f - width;
        double s = 0.0;
        for (int k = lane; k < width; k += 32) s = fma(band_b<BUILD>(B32, B64, e0 + k), xs[j0 + k], s);
        if (width > 1)
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const double S = __shfl_sync(0xffffffffu, s, 0);
        const double ic = ic_row[f];
        double X = S * ic;
        if (__double2hiint(ic) == 0 && __double2loint(ic) == 0) {
            X = 0.0;
            if (S != 0.0) numeric_bad = true;
        }
        if (lane == 0) xs[f] = X;
        total += X;
        bool stop = false;
        if (PRUNE) {  // the same test as k_recur, on lane-uniform values
            const int xe = ((__double2hiint(X) >> 20) & 0x7ff) + shift;
            const int ce = xe + kx[f];
            xmax = max(xmax, xe);
            cmax = max(cmax, ce);
            if (!(xe < xmax - L && ce < cmax - L)) last_big = f;
            stop = last_big < f - width;
        }
        if (above_rescale(X)) {
            __syncwarp();
            for (int i = lane; i <= f; i += 32) xs[i] *= kRescaleSmall;
            total *= kRescaleSmall;
            shift += 800;
        }
        __syncwarp();
        if (stop) {
            f_last = f;
            break;
        }
    }
    const double inv = 1.0 / total;
    double* prow = ch.P + (size_t)cell * ch.ldP + off;
    double emit = 0.0;
    for (int i = lane; i <= M; i += 32) {
        const double p = i <= f_last ? xs[i] * inv : 0.0;
        prow[i] = p;
        emit = fma(p, gd.cde[off + i], emit);
    }
    if (ch.ledger) {
        for (int o = 16; o > 0; o >>= 1) emit += __shfl_xor_sync(0xffffffffu, emit, o);
        if (lane == 0) {
            double* lg = ch.ledger + ((size_t)cell * gd.G + g) * 2;
            lg[0] = ch.pabs[(size_t)cell * gd.G + g];
            lg[1] = emit;
        }
    }
    if (numeric_bad && lane == 0) atomicOr(ch.status, kStatNumeric);
}

// ---------------------------------------------------------------------------
// Point-rule build (HEAT_HEATING_POINT; Eq. heating at the bin centres, Eq. brecurrence):
//   T_uj = Omega(lambda_uj) lambda_uj^3 dE_u / (h^2 c),  Omega(lambda) = u_n C_n e^{(su_n + sC_n) t}
// on the log-log interpolant (the slope of the product u C is the sum of the slopes), and
// B_uj = B_{u+1,j} + T_uj down each column from its last band row, in the order of the
// suffix recurrence.  Every band element is written (elements the rule leaves at zero
// carry the column's sum).  Also the absorbed power c int Omega on the grid, summed in
// k_build's order, for the energy check.
__device__ __forceinline__ double point_column(const GrainDev& gd, const ChunkDev& ch, int g, int cell, int j,
                                               double* Bb) {
    const int N = gd.N, Cc = ch.Cc;
    const double* Cact = gd.Cact + (size_t)g * N;
    const double* sC = gd.sC + (size_t)g * N;
    const int off = gd.bin_off[g];
    const int k1 = gd.pcol[off + j + 1];
    double acc = 0.0, om = 0.0, s = 0.0;
    int ncur = -1;
    for (int k = gd.pcol[off + j]; k < k1; ++k) {
        const PointEnt pe = gd.pent[k];
        if (pe.n >= 0) {
            if (pe.n != ncur) {  // entries move up the wavelength grid along a column
                ncur = pe.n;
                om = ch.ua64[(size_t)pe.n * Cc + cell] * Cact[pe.n];
                s = ch.su64[(size_t)pe.n * Cc + cell] + sC[pe.n];
            }
            acc += om * exp(s * pe.t) * pe.fac;
        }
        Bb[(size_t)pe.e * 32] = acc;
    }
    return acc;
}

__device__ __forceinline__ double absorbed_power(const GrainDev& gd, const ChunkDev& ch, int g, int cell) {
    const int N = gd.N, Cc = ch.Cc;
    const double* Cact = gd.Cact + (size_t)g * N;
    const double* sC = gd.sC + (size_t)g * N;
    double Psi = 0.0;
    for (int n = N - 2; n >= 0; --n) {
        const double om = ch.ua64[(size_t)n * Cc + cell] * Cact[n];
        const double q0 = ch.su64[(size_t)n * Cc + cell] + sC[n] + 1.0;
        const double b = om * gd.lam[n];
        const double dl = gd.dln[n];
        if (om > 0.0) Psi += b * dl * e1d(q0 * dl);
    }
    return kC * Psi;
}

// Lane per cell, warp per task (grain x 32 cells), columns in turn.
__global__ void __launch_bounds__(128) k_build_point(GrainDev gd, ChunkDev ch) {
    const int task = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (task >= ch.n_tasks) return;
    const int2 tk = (ch.btasks ? ch.btasks : ch.tasks)[task];
    const int g = tk.x, grp = tk.y;
    const int cell = grp * 32 + lane;
    const int M = gd.bin_off[g + 1] - gd.bin_off[g] - 1;
    double* Bb = ch.Bb64 + (size_t)grp * gd.band_total * 32 + lane;
    for (int j = 0; j < M; ++j) point_column(gd, ch, g, cell, j, Bb);
    if (ch.pabs) ch.pabs[(size_t)cell * gd.G + g] = absorbed_power(gd, ch, g, cell);
}

// Few cells: block per (cell, grain), threads over the columns (each column's sum is the
// same sequence as in k_build_point, so B is bit-identical).
__global__ void __launch_bounds__(128) k_build_point_small(GrainDev gd, ChunkDev ch) {
    const int cell = blockIdx.x / gd.G, g = blockIdx.x % gd.G;
    if (cell >= ch.cells) return;
    const int M = gd.bin_off[g + 1] - gd.bin_off[g] - 1;
    double* Bb = ch.Bb64 + (size_t)(cell >> 5) * gd.band_total * 32 + (cell & 31);
    for (int j = threadIdx.x; j < M; j += blockDim.x) point_column(gd, ch, g, cell, j, Bb);
    if (threadIdx.x == 0 && ch.pabs) ch.pabs[(size_t)cell * gd.G + g] = absorbed_power(gd, ch, g, cell);
}

// Blocks of 128 threads (a warp per task) for the task-list kernels: one per 4 tasks, or, for
// the persistent launches (ch.work set), no more than stay resident on the device at once.
template <typename K>
static unsigned task_grid(K kernel, const ChunkDev& ch) {
    const unsigned full = (unsigned)((ch.n_tasks + 3) / 4);
    if (!ch.work) return full;
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 128, 0) != cudaSuccess)
        return full;
    const unsigned cap = (unsigned)(sms > 0 && occ > 0 ? sms * occ : 1);
    return full < cap ? full : cap;
}

cudaError_t launch_field(const GrainDev& g, const void* u, int dtype, long long cell0, const ChunkDev& ch, int build,
                         cudaStream_t st) {
    dim3 block(32, 8), grid((g.N + 31) / 32, ch.Cc / 32);
    if (build == 0) {
        if (dtype == 0)
            k_field<double, double><<<grid, block, 0, st>>>(g.N, g.dln, (const double*)u, cell0, ch.cells, ch.Cc, ch.ua64,
                                                            ch.su64, ch.status);
        else
            k_field<float, double><<<grid, block, 0, st>>>(g.N, g.dln, (const float*)u, cell0, ch.cells, ch.Cc, ch.ua64,
                                                           ch.su64, ch.status);
    } else {
        if (dtype == 0)
            k_field<double, float><<<grid, block, 0, st>>>(g.N, g.dln, (const double*)u, cell0, ch.cells, ch.Cc, ch.ua32,
                                                           ch.su32, ch.status);
        else
            k_field<float, float><<<grid, block, 0, st>>>(g.N, g.dln, (const float*)u, cell0, ch.cells, ch.Cc, ch.ua32,
                                                          ch.su32, ch.status);
    }
    return cudaGetLastError();
}

cudaError_t launch_build(const GrainDev& g, const ChunkDev& ch, int build, cudaStream_t st) {
    if (ch.point) {  // the point rule (FP64 build only; checked by the caller)
        if (build != 0) return cudaErrorInvalidValue;
        if (ch.small) {
            const unsigned blocks = (unsigned)(ch.cells * g.G);
            if (blocks) k_build_point_small<<<blocks, 128, 0, st>>>(g, ch);
        } else {
            k_build_point<<<(ch.n_tasks + 3) / 4, 128, 0, st>>>(g, ch);
        }
        return cudaGetLastError();
    }
    if (ch.small) {
        const size_t smem = sizeof(double) * 2 * (size_t)g.N;
        const unsigned blocks = (unsigned)(ch.cells * g.G);
        if (blocks == 0) return cudaSuccess;
        if (smem > 48 * 1024) {
            cudaError_t e = build == 0 ? cudaFuncSetAttribute(k_build_small<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                              (int)smem)
                                       : cudaFuncSetAttribute(k_build_small<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                              (int)smem);
            if (e != cudaSuccess) return e;
        }
        if (build == 0)
            k_build_small<0><<<blocks, 256, smem, st>>>(g, ch);
        else
            k_build_small<1><<<blocks, 256, smem, st>>>(g, ch);
        return cudaGetLastError();
    }
    if (ch.n_tasks == 0) return cudaSuccess;
    // one warp per task: every task of a chunk fits on the device at once (39 registers,
    // up to 16 blocks per SM), so a persistent launch only adds the counter traffic
    ChunkDev c1 = ch;
    c1.work = nullptr;
    auto kern = build == 0 ? k_build<0> : k_build<1>;
    kern<<<task_grid(kern, c1), 128, 0, st>>>(g, c1);
    return cudaGetLastError();
}

cudaError_t launch_recur(const GrainDev& g, const ChunkDev& ch, int build, cudaStream_t st) {
    if (ch.small) {
        const long long warps = (long long)ch.cells * g.G;
        if (warps == 0) return cudaSuccess;
        const size_t smem = sizeof(double) * 4 * (size_t)g.max_bins;  // 4 warps per block
        auto kern = build == 0 ? (ch.prune ? k_recur_small<0, true> : k_recur_small<0, false>)
                               : (ch.prune ? k_recur_small<1, true> : k_recur_small<1, false>);
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        const unsigned blocks = (unsigned)((warps + 3) / 4);
        kern<<<blocks, 128, smem, st>>>(g, ch);
        return cudaGetLastError();
    }
    if (ch.n_tasks == 0) return cudaSuccess;
    auto kern = build == 0 ? (ch.prune ? k_recur<0, true> : k_recur<0, false>)
                           : (ch.prune ? k_recur<1, true> : k_recur<1, false>);
    kern<<<task_grid(kern, ch), 128, 0, st>>>(g, ch);
    return cudaGetLastError();
}

}  // namespace heat
