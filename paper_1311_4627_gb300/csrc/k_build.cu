// Per-solve kernels before the recursion: field tables (log-log slopes of u) and the matrix
// build (B band, Eq. bmatrix telescoped, intra-bin terms; or the point rule of Eq. heating
// with the suffix sums of Eq. brecurrence), as lane-per-cell kernels (warp = grain x 32 cells)
// and element-parallel kernels for solves of few cells.
#include <algorithm>

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
template <int BUILD, bool PF = false>
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
            const double dl = gd.dln[n];
            const int cls = series_class64(q1, dl);  // per cell, like the FP32 build's series choice
            if (cls == 2) {
                for (int k = sp[n]; k < sp[n + 1]; ++k) {
                    PatF64 pt = gd.pat64[k];
                    ch.Bb64[bb + (size_t)pt.e * 32] = Phi + (a * pt.t) * e1d_series_short(q1 * pt.t);
                }
                if (om > 0.0) Phi += a * dl * e1d_series_short(q1 * dl);
            } else if (cls == 1) {
                for (int k = sp[n]; k < sp[n + 1]; ++k) {
                    PatF64 pt = gd.pat64[k];
                    ch.Bb64[bb + (size_t)pt.e * 32] = Phi + (a * pt.t) * e1d_series(q1 * pt.t);
                }
                if (om > 0.0) Phi += a * dl * e1d_series(q1 * dl);
            } else {
                double aq = (q1 != 0.0) ? a / q1 : a;
                for (int k = sp[n]; k < sp[n + 1]; ++k) {
                    PatF64 pt = gd.pat64[k];
                    double B = Phi + (q1 != 0.0 ? aq * expm1(q1 * pt.t) : aq * pt.t);
                    ch.Bb64[bb + (size_t)pt.e * 32] = B;
                }
                if (om > 0.0) Phi += a * dl * e1d(q1 * dl);
            }
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
            // PF: L1 prefetch of the pattern line 32 entries past this segment (about three segments
            // ahead; the table is padded for it).  Measured on the batched workload (1024
            // wavelengths), A/B in one run: none 4.10 ms, 8 entries 3.93, 16 3.92, 32 3.87, 64 3.88,
            // 128 3.90, two lines 3.94; on the 2048-wavelength emissivity-heavy one it is slower
            // (70.5 -> 87.1 ms), so the host picks the variant per grid (heat_opts.build_prefetch)
            if (PF) asm volatile("prefetch.global.L1 [%0];" ::"l"(gd.pat32 + k1 + 32));
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

// One warp per task, in the build's task order.
template <int BUILD, bool PF = false>
__global__ void __launch_bounds__(128) k_build(GrainDev gd, ChunkDev ch) {
    const int task = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (task < ch.n_tasks) build_task<BUILD, PF>(gd, ch, task, threadIdx.x & 31);
}

// ---------------------------------------------------------------------------
// Element-parallel build for solves of few cells (ChunkDev::small): the same quantities as
// k_build with the same expressions; the cumulative sums run in the same order (one thread),
// so B is bit-identical.

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

// Blocks per (cell, grain): S parts (256 threads each, dynamic shared memory 2 N doubles).
// Every part forms the segment increments and the cumulative sums; part q writes the
// elements of the segments n = q (mod S), and the intra-bin terms whose diagonal element it
// wrote: the diagonal (j+1, j) and bin j's soft-photon edge are the same wavelength,
// hc/(Elo_{j+1} - E_j), so both fall in segment sf.n (sf.n < 0: the diagonal is not in the
// band, part 0).  Few spectra (a single cell) then spread over many SMs.
template <int BUILD>
__global__ void __launch_bounds__(256) k_build_small(GrainDev gd, ChunkDev ch, int S) {
    extern __shared__ double sm[];
    double* sPhi = sm;          // [N]: Phi before segment n (exclusive prefix), then Phi at the end
    double* sPsi = sm + gd.N;   // [N]: Psi after the segments above n (exclusive suffix)
    __shared__ double sPhiEnd, sPsiTot;
    __shared__ float sPsiEnd32;  // FP32 build: the FP32 value of the compensated total
    const int N = gd.N, Cc = ch.Cc;
    const int spec = blockIdx.x / S, part = blockIdx.x % S;
    const int cell = spec / gd.G, g = spec % gd.G;
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
                const int cls = series_class64(s.q1, s.dl);
                dphi = s.a * s.dl * (cls ? e1d_by_class(cls, s.q1 * s.dl) : e1d(s.q1 * s.dl));
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
    // (the increments are read eight at a time ahead of the sums, so no shared-memory load
    // latency sits on the sums' dependent chain)
    constexpr int R = 8;
    if (tid == 0) {
        if (BUILD == 0) {
            double Phi = 0.0;
            for (int n0 = 0; n0 < N - 1; n0 += R) {
                double d[R];
#pragma unroll
                for (int k = 0; k < R; ++k) d[k] = n0 + k < N - 1 ? sPhi[n0 + k] : 0.0;
#pragma unroll
                for (int k = 0; k < R; ++k)
                    if (n0 + k < N - 1) {
                        sPhi[n0 + k] = Phi;
                        Phi += d[k];
                    }
            }
            sPhiEnd = Phi;
        } else {
            Sum32 Phi;
            for (int n0 = 0; n0 < N - 1; n0 += R) {
                float d[R];
#pragma unroll
                for (int k = 0; k < R; ++k) d[k] = n0 + k < N - 1 ? (float)sPhi[n0 + k] : 0.0f;
#pragma unroll
                for (int k = 0; k < R; ++k)
                    if (n0 + k < N - 1) {
                        sPhi[n0 + k] = Phi.val();
                        Phi.add(d[k]);
                    }
            }
            sPhiEnd = Phi.val();
        }
    } else if (tid == 32) {
        if (BUILD == 0) {
            double Psi = 0.0;
            for (int n0 = N - 2; n0 >= 0; n0 -= R) {
                double d[R];
#pragma unroll
                for (int k = 0; k < R; ++k) d[k] = n0 - k >= 0 ? sPsi[n0 - k] : 0.0;
#pragma unroll
                for (int k = 0; k < R; ++k)
                    if (n0 - k >= 0) {
                        sPsi[n0 - k] = Psi;
                        Psi += d[k];
                    }
            }
            sPsiTot = Psi;
        } else {
            Sum32 Psi;
            for (int n0 = N - 2; n0 >= 0; n0 -= R) {
                float d[R];
#pragma unroll
                for (int k = 0; k < R; ++k) d[k] = n0 - k >= 0 ? (float)sPsi[n0 - k] : 0.0f;
#pragma unroll
                for (int k = 0; k < R; ++k)
                    if (n0 - k >= 0) {
                        sPsi[n0 - k] = Psi.val();
                        Psi.add(d[k]);
                    }
            }
            sPsiTot = Psi.wide();
            sPsiEnd32 = Psi.val();
        }
    }
    __syncthreads();
    // 3. band elements: warp per segment (this part's), lanes over its pattern entries
    for (int n = part + S * warp; n < N - 1; n += S * (blockDim.x >> 5)) {
        const int k0 = sp[n], k1 = sp[n + 1];
        if (k0 == k1) continue;
        if (BUILD == 0) {
            const SegF64 s = seg64(gd, g, n, ch.ua64[(size_t)n * Cc + cell], ch.su64[(size_t)n * Cc + cell]);
            const double aq = (s.q1 != 0.0) ? s.a / s.q1 : s.a;
            const double Phi = sPhi[n];
            const int cls = series_class64(s.q1, s.dl);
            for (int k = k0 + lane; k < k1; k += 32) {
                const PatF64 pt = gd.pat64[k];
                ch.Bb64[bb + (size_t)pt.e * 32] =
                    cls ? Phi + (s.a * pt.t) * e1d_by_class(cls, s.q1 * pt.t)
                        : Phi + (s.q1 != 0.0 ? aq * expm1(s.q1 * pt.t) : aq * pt.t);
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
    if ((N - 1) % S == part)
        for (int k = sp[N - 1] + tid; k < sp[N]; k += blockDim.x) {
            if (BUILD == 0)
                ch.Bb64[bb + (size_t)gd.pat64[k].e * 32] = sPhiEnd;
            else
                ch.Bb32[bb + (size_t)gd.pat32[k].e * 32] = __double2float_rn(sPhiEnd);
        }
    __syncthreads();  // the intra-bin terms add to diagonal elements written above (by this part)
    // 4. intra-bin terms, one per soft entry (each has its own diagonal element)
    for (int p = gd.soft_off[g] + tid; p < gd.soft_off[g + 1]; p += blockDim.x) {
        const SoftF64 sf = gd.soft[p];
        if ((sf.n < 0 ? 0 : sf.n % S) != part) continue;
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
    if (tid == 0 && part == 0 && ch.pabs) ch.pabs[(size_t)cell * gd.G + g] = BUILD == 0 ? kC * sPsiTot : sPsiTot;
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
    bool ser = false;
    int ncur = -1;
    for (int k = gd.pcol[off + j]; k < k1; ++k) {
        const PointEnt pe = gd.pent[k];
        if (pe.n >= 0) {
            if (pe.n != ncur) {  // entries move up the wavelength grid along a column
                ncur = pe.n;
                om = ch.ua64[(size_t)pe.n * Cc + cell] * Cact[pe.n];
                s = ch.su64[(size_t)pe.n * Cc + cell] + sC[pe.n];
                ser = short_series64(s, gd.dln[pe.n]);
            }
            const double z = s * pe.t;  // e^z = 1 + z E1(z)
            acc += om * (ser ? fma(z, e1d_series(z), 1.0) : exp(z)) * pe.fac;
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
        const long long spectra = (long long)ch.cells * g.G;
        if (spectra == 0) return cudaSuccess;
        // parts per spectrum: about two blocks per SM in all (one part when spectra suffice)
        int dev = 0, sms = 152;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int S = (int)std::max(1LL, std::min(16LL, 2LL * sms / spectra));
        const unsigned blocks = (unsigned)(spectra * S);
        if (smem > 48 * 1024) {
            cudaError_t e = build == 0 ? cudaFuncSetAttribute(k_build_small<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                              (int)smem)
                                       : cudaFuncSetAttribute(k_build_small<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                              (int)smem);
            if (e != cudaSuccess) return e;
        }
        if (build == 0)
            k_build_small<0><<<blocks, 256, smem, st>>>(g, ch, S);
        else
            k_build_small<1><<<blocks, 256, smem, st>>>(g, ch, S);
        return cudaGetLastError();
    }
    if (ch.n_tasks == 0) return cudaSuccess;
    // one warp per task (measured: a persistent launch with a task counter is no faster)
    auto kern = build == 0 ? k_build<0> : (g.pat_prefetch ? k_build<1, true> : k_build<1, false>);
    kern<<<(unsigned)((ch.n_tasks + 3) / 4), 128, 0, st>>>(g, ch);
    return cudaGetLastError();
}

}  // namespace heat
