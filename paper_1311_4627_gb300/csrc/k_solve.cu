// Per-solve kernels: field tables, wavelength prefix tables, and the
// Guhathakurta-Draine recursion (Eq. bmatrix, Eq. xf, Eq. renormalization).
//
// Work unit ("task") = one grain x 32 cells; one warp per task, one lane per cell.
// All lanes of a warp walk the same band of the same grain, so the recursion has
// no divergence and no cross-lane reduction: each band element costs one FP64 FMA
// per cell.
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
            ua[(size_t)n * Cc + c] = t_ua[tx][ty + 8 * k];
            su[(size_t)n * Cc + c] = t_su[tx][ty + 8 * k];
        }
    }
    if (bad) atomicOr(status, kStatBadInput);
}

// ---------------------------------------------------------------------------
// k_prep (FP64 build).  Per cell and grain, with Omega = u C on the log-log
// interpolant (Eq. interpolation), slope s_n and q = s_n + p + 1:
//   segment integral   int Omega lambda^p = Omega_n lambda_n^{p+1} dln_n E1(q dln_n)
//   photon prefix      Phi_n = (1/h) sum_{m<n} int_m Omega lambda          (B_fj = Phi(lambda_fj))
//   element constants  aq_n = (Omega_n lambda_n^2/h)/q_n,  q_n  (q_n = 0: aq_n = Omega_n lambda_n^2/h)
//   intra-bin term     W_j = c int_{hc/(Elo_{j+1}-E_j)}^{lambda_{N-1}} Omega,  intra_j = W_j/(E_{j+1}-E_j)
//   absorbed power     c int Omega over the grid
__global__ void k_prep64(GrainDev gd, ChunkDev ch) {
    int task = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (task >= ch.n_tasks) return;
    const int N = gd.N, Cc = ch.Cc, nbt = gd.nbt;
    int g = ch.tasks[task].x, grp = ch.tasks[task].y;
    int off = gd.bin_off[g];
    const double* Cact = gd.Cact + (size_t)g * N;
    const double* sC = gd.sC + (size_t)g * N;
    int cc = grp * 32 + lane;
    size_t tb = (size_t)task * N * 32 + lane;
    size_t ib = ((size_t)grp * nbt + off) * 32 + lane;

    double Phi = 0.0;
    for (int n = 0; n < N - 1; ++n) {
        double ua = ch.ua64[(size_t)n * Cc + cc], su = ch.su64[(size_t)n * Cc + cc];
        double om = ua * Cact[n];
        double q1 = su + sC[n] + 2.0;
        double ln = gd.lam[n];
        double a = om * ln * ln / kH;
        ch.phi64[tb + (size_t)n * 32] = Phi;
        ch.aq64[tb + (size_t)n * 32] = (q1 != 0.0) ? a / q1 : a;
        ch.q64[tb + (size_t)n * 32] = q1;
        if (om > 0.0) Phi += a * gd.dln[n] * e1d(q1 * gd.dln[n]);
    }
    ch.phi64[tb + (size_t)(N - 1) * 32] = Phi;
    ch.aq64[tb + (size_t)(N - 1) * 32] = 0.0;
    ch.q64[tb + (size_t)(N - 1) * 32] = 0.0;

    const SoftF64* soft = gd.soft;
    int p = gd.soft_off[g], p1 = gd.soft_off[g + 1];
    while (p < p1 && soft[p].n == N - 1) {
        ch.intra64[ib + (size_t)soft[p].j * 32] = 0.0;
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
            ch.intra64[ib + (size_t)sf.j * 32] = kC * (part + Psi) * gd.invdE[off + sf.j];
            ++p;
        }
        if (om > 0.0) Psi += b * dl * e1d(q0 * dl);
    }
    for (; p < p1; ++p) ch.intra64[ib + (size_t)soft[p].j * 32] = kC * Psi * gd.invdE[off + soft[p].j];
    if (ch.pabs) ch.pabs[(size_t)cc * gd.G + g] = kC * Psi;
}

// k_prep (FP32 build): the photon prefix Phi_n and the intra-bin terms, in FP32 with
// compensated (Kahan) running sums.  The element constants are formed in the
// recursion from the shared field tables ua, su and the grain's ca, sC.
__global__ void k_prep32(GrainDev gd, ChunkDev ch) {
    int task = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (task >= ch.n_tasks) return;
    const int N = gd.N, Cc = ch.Cc, nbt = gd.nbt;
    int g = ch.tasks[task].x, grp = ch.tasks[task].y;
    int off = gd.bin_off[g];
    const float* ca = gd.ca32 + (size_t)g * N;
    const float* ce = gd.ce32 + (size_t)g * N;
    const float* sC = gd.sC32 + (size_t)g * N;
    int cc = grp * 32 + lane;
    size_t tb = (size_t)task * N * 32 + lane;
    size_t ib = ((size_t)grp * nbt + off) * 32 + lane;

    float Phi = 0.0f, cPhi = 0.0f;
    for (int n = 0; n < N - 1; ++n) {
        float ua = ch.ua32[(size_t)n * Cc + cc], su = ch.su32[(size_t)n * Cc + cc];
        ch.phi32[tb + (size_t)n * 32] = Phi;
        float a = ua * ca[n];
        if (a > 0.0f) {
            float dl = gd.dln32[n];
            float I = a * dl * e1f((su + sC[n] + 2.0f) * dl);
            float y = I - cPhi, t = Phi + y;
            cPhi = (t - Phi) - y;
            Phi = t;
        }
    }
    ch.phi32[tb + (size_t)(N - 1) * 32] = Phi;

    const SoftF64* soft = gd.soft;
    int p = gd.soft_off[g], p1 = gd.soft_off[g + 1];
    while (p < p1 && soft[p].n == N - 1) {
        ch.intra32[ib + (size_t)soft[p].j * 32] = 0.0f;
        ++p;
    }
    float Psi = 0.0f, cPsi = 0.0f;  // c int Omega from lambda_{n+1} to lambda_{N-1}
    for (int n = N - 2; n >= 0; --n) {
        float ua = ch.ua32[(size_t)n * Cc + cc], su = ch.su32[(size_t)n * Cc + cc];
        float b = ua * ce[n];
        float q0 = su + sC[n] + 1.0f;
        float dl = gd.dln32[n];
        while (p < p1 && soft[p].n == n) {
            SoftF64 sf = soft[p];
            float part = 0.0f;
            if (b > 0.0f) {
                float ts = (float)sf.t;
                float L = dl - ts;
                part = b * expf(q0 * ts) * L * e1f(q0 * L);
            }
            ch.intra32[ib + (size_t)sf.j * 32] = (part + Psi) * gd.invdE32[off + sf.j];
            ++p;
        }
        if (b > 0.0f) {
            float I = b * dl * e1f(q0 * dl);
            float y = I - cPsi, t = Psi + y;
            cPsi = (t - Psi) - y;
            Psi = t;
        }
    }
    for (; p < p1; ++p) ch.intra32[ib + (size_t)soft[p].j * 32] = Psi * gd.invdE32[off + soft[p].j];
    if (ch.pabs) ch.pabs[(size_t)cc * gd.G + g] = (double)Psi;
}

// ---------------------------------------------------------------------------
// k_recur: X_0 = 1, X_f = (sum_{j in band(f)} B_fj X_j + intra_{f-1} X_{f-1}) / T_{f-1,f}
// (Eq. xf; the band holds every j whose transition wavelength lies on the grid, all
// other B_fj are exactly zero), power-of-two rescale of X_0..X_f when X_f > 2^800,
// then P = X / sum X (Eq. renormalization) written to P[cell][off_g + i].
template <int BUILD>
__global__ void __launch_bounds__(128) k_recur(GrainDev gd, ChunkDev ch) {
    int task = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (task >= ch.n_tasks) return;
    const int N = gd.N, Cc = ch.Cc, nbt = gd.nbt;
    int g = ch.tasks[task].x, grp = ch.tasks[task].y;
    int off = gd.bin_off[g];
    int M = gd.bin_off[g + 1] - off - 1;
    int cc = grp * 32 + lane;
    size_t tb = (size_t)task * N * 32 + lane;
    size_t xb = ((size_t)grp * nbt + off) * 32 + lane;
    const int* rp = gd.rowptr + off + g;
    double* xs = ch.xs;
    bool numeric_bad = false;

    xs[xb] = 1.0;
    for (int f = 1; f <= M; ++f) {
        int e0 = rp[f], e1 = rp[f + 1];
        int j = f - (e1 - e0);
        double S = 0.0;
        if (BUILD == 0) {
#pragma unroll 2
            for (int e = e0; e < e1; ++e, ++j) {
                ElemF64 el = gd.el64[e];
                size_t ti = tb + (size_t)el.n * 32;
                double ph = ch.phi64[ti], aq = ch.aq64[ti], q = ch.q64[ti];
                double B = ph + (q != 0.0 ? aq * expm1(q * el.t) : aq * el.t);
                S = fma(B, xs[xb + (size_t)j * 32], S);
            }
            S = fma(ch.intra64[xb + (size_t)(f - 1) * 32], xs[xb + (size_t)(f - 1) * 32], S);
        } else {
#pragma unroll 4
            for (int e = e0; e < e1; ++e, ++j) {
                ElemF32 el = gd.el32[e];
                size_t fi = (size_t)el.n * Cc + cc;
                float ph = ch.phi32[tb + (size_t)el.n * 32];
                float ua = ch.ua32[fi], su = ch.su32[fi];
                float B = fmaf(ua * el.cat, e1f(fmaf(su, el.t, el.zt)), ph);
                S = fma(widen_pos(B), xs[xb + (size_t)j * 32], S);
            }
            S = fma(widen_pos(ch.intra32[xb + (size_t)(f - 1) * 32]), xs[xb + (size_t)(f - 1) * 32], S);
        }
        double ic = gd.invC[off + f];
        double X = S * ic;
        if (!(ic > 0.0)) {
            X = 0.0;
            if (S != 0.0) numeric_bad = true;
        }
        xs[xb + (size_t)f * 32] = X;
        if (X > kRescaleBig)
            for (int i = 0; i <= f; ++i) xs[xb + (size_t)i * 32] *= kRescaleSmall;
    }
    double sum = 0.0;
    for (int i = 0; i <= M; ++i) sum += xs[xb + (size_t)i * 32];
    double inv = 1.0 / sum;
    if (cc < ch.cells) {
        double* prow = ch.P + (size_t)cc * ch.ldP + off;
        for (int i = 0; i <= M; ++i) prow[i] = xs[xb + (size_t)i * 32] * inv;
    }
    if (numeric_bad) atomicOr(ch.status, kStatNumeric);
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

cudaError_t launch_prep(const GrainDev& g, const ChunkDev& ch, int build, cudaStream_t st) {
    int threads = 128, blocks = (ch.n_tasks + 3) / 4;
    if (build == 0)
        k_prep64<<<blocks, threads, 0, st>>>(g, ch);
    else
        k_prep32<<<blocks, threads, 0, st>>>(g, ch);
    return cudaGetLastError();
}

cudaError_t launch_recur(const GrainDev& g, const ChunkDev& ch, int build, cudaStream_t st) {
    int threads = 128, blocks = (ch.n_tasks + 3) / 4;
    if (build == 0)
        k_recur<0><<<blocks, threads, 0, st>>>(g, ch);
    else
        k_recur<1><<<blocks, threads, 0, st>>>(g, ch);
    return cudaGetLastError();
}

}  // namespace heat
