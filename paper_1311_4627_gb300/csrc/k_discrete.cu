// Thermal-discrete cooling (the approximation named beside Eq. adjacent) on the exact path:
// downward rates to every lower bin, and the stationary state of the full rate matrix
// (Eq. steady-state with Eq. level-sum) instead of the Guhathakurta-Draine recursion, which
// needs the adjacent-only cooling of Eq. adjacent.
//
//   k_cooling_window  (grain set-up, once): T_lu = P_emit(T_u; window of l) / (E_u - E_l),
//       the power of Eq. cooling's integrand at T_u in the photon energies that take a grain
//       from bin u to bin l, E in [E_u - Ehi_l, E_u - Elo_l] (l = u-1: [0, E_u - Elo_{u-1}],
//       photons too soft to leave bin u included); the windows tile [0, E_u], so the rates
//       carry the power Eq. cooling's adjacent rate carries.
//   k_td_fill  (per spectrum): the rate matrix q[i][j] (from i to j): heating elements
//       T_ji, j > i, as closed-form integrals over the target bin's wavelength window of the
//       log-log interpolant of Omega = u C (plus the intra-bin term on j = i + 1), downward
//       rates from the grain's table; and the absorbed power for the energy check.
//   k_gth  (per spectrum): state reduction (Grassmann, Taksar, Heyman): states n = M..1 are
//       removed, their rates redistributed, q_ij += q_in q_nj / s_n with s_n = sum_{j<n} q_nj
//       (sums and products of non-negative numbers only); then X_0 = 1,
//       X_n = sum_{i<n} X_i q_in / s_n, power-of-two rescales, P = X / sum X.  O(M^3) per
//       spectrum: meant for solves of few cells (one block per spectrum, q in device memory).
#include "common.cuh"
#include "internal.h"

namespace heat {

namespace {

constexpr double kPi = 3.141592653589793;

// Gauss-Legendre (the set-up's nodes, shared with k_cooling) over [ya, yb] in ln(lambda) of
// C(lambda) B_lambda(T) lambda with C = c0 (lambda/lam0)^s.
__device__ double gl_panel(double ya, double yb, double c0, double lam0, double s, double T, const double* glx,
                           const double* glw) {
    double m = 0.5 * (ya + yb), r = 0.5 * (yb - ya), acc = 0.0;
    for (int k = 0; k < kGLPoints; ++k) {
        const double lam = exp(m + r * glx[k]);
        const double x = kHC / (lam * kK * T);
        if (x > 745.0) continue;
        const double l2 = lam * lam;
        const double bl = 2.0 * kH * kC * kC / (l2 * l2 * lam) / expm1(x);
        acc += glw[k] * c0 * pow(lam / lam0, s) * bl * lam;
    }
    return acc * r;
}

// The same over [ya, yb] in sub-panels short enough for the Wien factor: d ln(integrand) /
// d ln(lambda) is about x - 4 + s with x = hc/(lambda k T), so a step of 2/max(x, 4) in
// ln(lambda) keeps each sub-panel within a few e-folds, and every window, however far into the
// tail, is integrated to its own relative accuracy.
__device__ double window_panel(double ya, double yb, double c0, double lam0, double s, double T,
                               const double* glx, const double* glw) {
    double acc = 0.0;
    for (double y = ya; y < yb;) {
        const double x = kHC / (exp(y) * kK * T);
        double h = 2.0 / fmax(x, 4.0);
        if (h > 0.25) h = 0.25;
        const double y1 = y + h < yb ? y + h : yb;
        acc += gl_panel(y, y1, c0, lam0, s, T, glx, glw);
        y = y1;
    }
    return acc;
}

// C(lambda): the log-log interpolant of the nodes, continued beyond the grid with the end
// segments' power laws (as the cooling integral takes it).
__device__ double cabs_at(int N, const double* lam, const double* C, double x) {
    int n;
    if (x < lam[0]) {
        n = 0;
    } else {
        int lo = 0, hi = N - 2;  // last segment with lam[n] <= x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (lam[mid] <= x) lo = mid; else hi = mid - 1;
        }
        n = lo;
    }
    if (!(C[n] > 0.0 && C[n + 1] > 0.0)) return 0.0;
    return C[n] * pow(x / lam[n], log(C[n + 1] / C[n]) / log(lam[n + 1] / lam[n]));
}

// A narrow window written in the grain's energy after the emission, e in [e0, e0 + de]
// (photon energy E_u - e): its width is exact where it is a tiny fraction of the photon
// energy, which a difference of photon-energy limits would lose.  Gauss-Legendre pieces
// between the grid nodes inside.  Returns int C(E) E^3 / (e^(E/kT) - 1) dE over the window.
__device__ double narrow_window(int N, const double* lam, const double* C, double T, double Eu, double e0, double de,
                                const double* glx, const double* glw) {
    // nodes inside: photon energies hc/lam_n in (Eu - e0 - de, Eu - e0)
    double cuts[6];
    int nc = 0;
    cuts[nc++] = 0.0;
    for (int n = 0; n < N && nc < 5; ++n) {
        const double o = (Eu - kHC / lam[n]) - e0;
        if (o > 0.0 && o < de) cuts[nc++] = o;
    }
    cuts[nc++] = de;
    for (int i = 1; i < nc; ++i) {  // ascending
        const double v = cuts[i];
        int k = i - 1;
        while (k >= 0 && cuts[k] > v) {
            cuts[k + 1] = cuts[k];
            --k;
        }
        cuts[k + 1] = v;
    }
    double acc = 0.0;
    for (int i = 0; i + 1 < nc; ++i) {
        const double r = 0.5 * (cuts[i + 1] - cuts[i]), m = cuts[i] + r;
        if (!(r > 0.0)) continue;
        double s = 0.0;
        for (int k = 0; k < kGLPoints; ++k) {
            const double eps = Eu - (e0 + m + r * glx[k]);
            const double x = eps / (kK * T);
            if (!(eps > 0.0) || x > 745.0) continue;
            s += glw[k] * cabs_at(N, lam, C, kHC / eps) * eps * eps * eps / expm1(x);
        }
        acc += s * r;
    }
    return acc;
}

}  // namespace

// One warp per window (grain g, upper bin u, lower bin l < u); windows of grain g are
// numbered k = u(u-1)/2 + l from woff[g].  Panels as k_cooling's (each grid segment, and
// 0.25 in ln(lambda) beyond the grid with the end segments' power laws), clipped to the
// window's wavelengths [hc/Emax, hc/Emin].
__global__ void k_cooling_window(int N, const double* __restrict__ lam, const double* __restrict__ cabs,
                                 const int* __restrict__ bin_off, int G, const double* __restrict__ T,
                                 const double* __restrict__ E, const long long* __restrict__ woff,
                                 const long long* __restrict__ doff, double* __restrict__ D, const double* glx,
                                 const double* glw) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= woff[G]) return;
    int g = 0;
    {
        int lo = 0, hi = G - 1;  // last g with woff[g] <= w
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (woff[mid] <= w) lo = mid; else hi = mid - 1;
        }
        g = lo;
    }
    const long long k = w - woff[g];
    int u = (int)floor((1.0 + sqrt(1.0 + 8.0 * (double)k)) * 0.5);
    while ((long long)u * (u - 1) / 2 > k) --u;
    while ((long long)(u + 1) * u / 2 <= k) ++u;
    const int l = (int)(k - (long long)u * (u - 1) / 2);
    const int off = bin_off[g], nb = bin_off[g + 1] - off;
    const double* Eg = E + off;
    const double Tu = T[off + u];
    const double elo_l = l == 0 ? 0.0 : 0.5 * (Eg[l - 1] + Eg[l]);
    const double ehi_l = 0.5 * (Eg[l] + Eg[l + 1]);
    const double emin = l == u - 1 ? 0.0 : Eg[u] - ehi_l;
    const double emax = Eg[u] - elo_l;
    // wavelengths of the window, cut where the integrand is below 1e-340 of its scale
    double lo = kHC / emax;
    const double lmin = kHC / (800.0 * kK * Tu);
    if (lo < lmin) lo = lmin;
    const double hi = emin > 0.0 ? kHC / emin : INFINITY;
    const double* C = cabs + (size_t)g * N;
    if (l < u - 1 && ehi_l - elo_l < 1e-2 * emin) {  // narrow: in the grain's final energy
        if (lane == 0) {
            const double p = 8.0 * kPi / (kH * kH * kH * kC * kC) *
                             narrow_window(N, lam, C, Tu, Eg[u], elo_l, ehi_l - elo_l, glx, glw);
            D[doff[g] + (size_t)l * nb + u] = p / (Eg[u] - Eg[l]);
        }
        return;
    }
    double acc = 0.0;
    if (hi > lo) {
        for (int n = lane; n < N - 1; n += 32) {  // grid segments
            const double a = lam[n], b = lam[n + 1];
            if (b <= lo || a >= hi || !(C[n] > 0.0 && C[n + 1] > 0.0)) continue;
            const double s = log(C[n + 1] / C[n]) / log(b / a);
            acc += window_panel(log(a > lo ? a : lo), log(b < hi ? b : hi), C[n], a, s, Tu, glx, glw);
        }
        if (C[N - 2] > 0.0 && C[N - 1] > 0.0 && hi > lam[N - 1]) {  // past the last node
            const double s = log(C[N - 1] / C[N - 2]) / log(lam[N - 1] / lam[N - 2]);
            const double y0 = log(lam[N - 1] > lo ? lam[N - 1] : lo);
            const double y1 = hi < INFINITY ? log(hi) : y0 + 25.0;
            for (int k2 = lane; y0 + 0.25 * k2 < y1; k2 += 32) {
                const double yb = y0 + 0.25 * (k2 + 1);
                acc += window_panel(y0 + 0.25 * k2, yb < y1 ? yb : y1, C[N - 1], lam[N - 1], s, Tu, glx, glw);
            }
        }
        if (lo < lam[0] && C[0] > 0.0 && C[1] > 0.0) {  // below the first node
            const double s = log(C[1] / C[0]) / log(lam[1] / lam[0]);
            const double ytop = log(hi < lam[0] ? hi : lam[0]), ybot = log(lo);
            for (int k2 = lane; ytop - 0.25 * k2 > ybot; k2 += 32) {
                const double yb = ytop - 0.25 * k2;
                double ya = yb - 0.25;
                if (ya < ybot) ya = ybot;
                acc += window_panel(ya, yb, C[0], lam[0], s, Tu, glx, glw);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) D[doff[g] + (size_t)l * nb + u] = 4.0 * kPi * acc / (Eg[u] - Eg[l]);
}

namespace {

// Integral over [x, y] of Omega lambda^p in segment n of the cell's interpolant:
// Omega_n lambda_n^(p+1) e^(q tx) (ty - tx) E1(q (ty - tx)), q = s_n + p + 1.
__device__ __forceinline__ double seg_part(double om, double s, double lamn, int p, double x, double y) {
    const double tx = log(x / lamn), dt = log(y / x);
    const double q = s + p + 1.0;
    const double lp = p == 1 ? lamn * lamn : lamn;
    return om * lp * exp(q * tx) * dt * e1d(q * dt);
}

// Integral of Omega lambda^p over [a, b] (clipped to the grid) for one cell and grain.
__device__ double range_integral(const GrainDev& gd, const ChunkDev& ch, int g, int cell, int p, double a, double b) {
    const int N = gd.N;
    const double* lam = gd.lam;
    if (a < lam[0]) a = lam[0];
    if (b > lam[N - 1]) b = lam[N - 1];
    if (!(b > a)) return 0.0;
    int n = 0;
    {
        int lo = 0, hi = N - 2;  // last segment with lam[n] <= a
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (lam[mid] <= a) lo = mid; else hi = mid - 1;
        }
        n = lo;
    }
    double acc = 0.0;
    for (; n < N - 1 && lam[n] < b; ++n) {
        const double om = ch.ua64[(size_t)n * ch.Cc + cell] * gd.Cact[(size_t)g * N + n];
        if (!(om > 0.0)) continue;
        const double s = ch.su64[(size_t)n * ch.Cc + cell] + gd.sC[(size_t)g * N + n];
        const double x = lam[n] > a ? lam[n] : a, y = lam[n + 1] < b ? lam[n + 1] : b;
        if (y > x) acc += seg_part(om, s, lam[n], p, x, y);
    }
    return acc;
}

}  // namespace

// One block per spectrum (cell, grain) of the chunk's cells: q [nb][nb] (row-major, rate from
// row to column) at q + spectrum * qstride; the absorbed power c int Omega on the grid.
__global__ void __launch_bounds__(256) k_td_fill(GrainDev gd, ChunkDev ch, const double* __restrict__ D,
                                                 const long long* __restrict__ doff, long long s0, double* q,
                                                 long long qstride) {
    const long long sp = s0 + blockIdx.x;
    const int cell = (int)(sp / gd.G), g = (int)(sp % gd.G);
    const int off = gd.bin_off[g], nb = gd.bin_off[g + 1] - off;
    const double* E = gd.E + off;
    const double* Dg = D + doff[g];
    double* qs = q + (size_t)blockIdx.x * qstride;
    for (long long idx = threadIdx.x; idx < (long long)nb * nb; idx += blockDim.x) {
        const int i = (int)(idx / nb), j = (int)(idx % nb);
        double v = 0.0;
        if (j < i) {
            v = Dg[(size_t)j * nb + i];
        } else if (j > i) {  // heating from i into bin j: photons of [Elo_j - E_i, Ehi_j - E_i)
            const int M = nb - 1;
            const double elo = 0.5 * (E[j - 1] + E[j]);
            const double la = j == M ? 0.0 : kHC / (0.5 * (E[j] + E[j + 1]) - E[i]);
            const double lb = kHC / (elo - E[i]);
            v = range_integral(gd, ch, g, cell, 1, la, lb) / kH;
            if (j == i + 1)  // photons too soft to leave bin i (their power, per transition energy)
                v += kC * range_integral(gd, ch, g, cell, 0, lb, gd.lam[gd.N - 1]) / (E[j] - E[i]);
        }
        qs[idx] = v;
    }
    if (threadIdx.x == 0 && ch.pabs)
        ch.pabs[(size_t)cell * gd.G + g] = kC * range_integral(gd, ch, g, cell, 0, gd.lam[0], gd.lam[gd.N - 1]);
}

namespace {

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) red[0] = t;
    }
    __syncthreads();
    return red[0];
}

}  // namespace

// One block per spectrum: state reduction of q, back substitution, P and the energy check.
// Shared memory: s[nb] (exit rates), r[nb] (the removed state's rates / s_n), X[nb].
__global__ void __launch_bounds__(256) k_gth(GrainDev gd, ChunkDev ch, long long s0, double* q, long long qstride) {
    extern __shared__ double smd[];
    __shared__ double red[8];
    const long long sp = s0 + blockIdx.x;
    const int cell = (int)(sp / gd.G), g = (int)(sp % gd.G);
    const int off = gd.bin_off[g], nb = gd.bin_off[g + 1] - off;
    double* qs = q + (size_t)blockIdx.x * qstride;
    double* s = smd;
    double* r = smd + nb;
    double* X = smd + 2 * nb;
    for (int n = nb - 1; n >= 1; --n) {
        double part = 0.0;
        for (int j = threadIdx.x; j < n; j += blockDim.x) part += qs[(size_t)n * nb + j];
        const double sn = block_sum(part, red);
        if (threadIdx.x == 0) s[n] = sn;
        if (sn == 0.0) continue;  // uniform: nothing leaves n downward
        for (int j = threadIdx.x; j < n; j += blockDim.x) r[j] = qs[(size_t)n * nb + j] / sn;
        __syncthreads();
        for (long long idx = threadIdx.x; idx < (long long)n * n; idx += blockDim.x) {
            const int i = (int)(idx / n), j = (int)(idx % n);
            const double qin = qs[(size_t)i * nb + n];
            if (i != j && qin != 0.0) qs[(size_t)i * nb + j] = fma(qin, r[j], qs[(size_t)i * nb + j]);
        }
        __syncthreads();
    }
    // back substitution (X in shared memory), rescaled by 2^-800 past 2^800
    if (threadIdx.x == 0) X[0] = 1.0;
    __syncthreads();
    double total = 1.0;
    bool bad = false;
    for (int n = 1; n < nb; ++n) {
        double part = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) part += X[i] * qs[(size_t)i * nb + n];
        const double in = block_sum(part, red);
        const double sn = s[n];
        double xn = 0.0;
        if (sn == 0.0) {
            if (in != 0.0) bad = true;
        } else {
            xn = in / sn;
        }
        total += xn;
        if (xn > 0x1p800) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) X[i] *= 0x1p-800;
            xn *= 0x1p-800;
            total *= 0x1p-800;
        }
        if (threadIdx.x == 0) X[n] = xn;
        __syncthreads();
    }
    const double inv = 1.0 / total;
    double emit = 0.0;
    if (cell < ch.cells) {
        double* prow = ch.P + (size_t)cell * ch.ldP + off;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            const double p = X[i] * inv;
            prow[i] = p;
            emit = fma(p, gd.cde[off + i], emit);
        }
    }
    emit = block_sum(emit, red);
    if (threadIdx.x == 0 && cell < ch.cells) {
        if (ch.ledger) {
            double* lg = ch.ledger + ((size_t)cell * gd.G + g) * 2;
            lg[0] = ch.pabs[(size_t)cell * gd.G + g];
            lg[1] = emit;
        }
        if (bad) atomicOr(ch.status, kStatNumeric);
    }
}

cudaError_t launch_cooling_window(int N, const double* lam, const double* cabs, const int* bin_off, int G,
                                  const double* T, const double* E, const long long* woff, long long n_windows,
                                  const long long* doff, double* D, const double* glx, const double* glw,
                                  cudaStream_t st) {
    if (n_windows <= 0) return cudaSuccess;
    const long long threads = n_windows * 32;
    k_cooling_window<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(N, lam, cabs, bin_off, G, T, E, woff, doff,
                                                                        D, glx, glw);
    return cudaGetLastError();
}

cudaError_t launch_discrete_solve(const GrainDev& g, const ChunkDev& ch, const double* D, const long long* doff,
                                  double* q, long long qstride, long long batch, cudaStream_t st) {
    const long long spectra = (long long)ch.cells * g.G;
    const size_t smem = sizeof(double) * 3 * (size_t)g.max_bins;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_gth, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    for (long long s0 = 0; s0 < spectra; s0 += batch) {
        const unsigned n = (unsigned)(spectra - s0 < batch ? spectra - s0 : batch);
        k_td_fill<<<n, 256, 0, st>>>(g, ch, D, doff, s0, q, qstride);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_gth<<<n, 256, smem, st>>>(g, ch, s0, q, qstride);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace heat
