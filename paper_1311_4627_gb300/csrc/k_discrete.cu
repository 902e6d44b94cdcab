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
//       X_n = sum_{i<n} X_i q_in / s_n, power-of-two rescales, P = X / sum X.  About M^3/3
//       fused multiply-adds per spectrum, on the FP64 unit: one block per spectrum, states
//       removed eight at a time with one delayed rank-8 update of the rest (q in shared memory
//       up to 160 bins, else in device memory, read and written once per eight states).
#include <algorithm>

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
            D[doff[g] + (size_t)u * nb + l] = p / (Eg[u] - Eg[l]);
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
    if (lane == 0) D[doff[g] + (size_t)u * nb + l] = 4.0 * kPi * acc / (Eg[u] - Eg[l]);
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

// Segment n (0 .. N-2) holding x in [lam_0, lam_{N-1}]: lam_n <= x < lam_{n+1} (x = lam_{N-1} in
// the last).  Searched in FP32, then moved by at most one node with the FP64 grid.
__device__ __forceinline__ int seg_of(const float* l32, const double* lam, int N, double x) {
    const float xf = (float)x;
    int lo = 0, hi = N - 2;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (l32[mid] <= xf) lo = mid; else hi = mid - 1;
    }
    if (lo < N - 2 && lam[lo + 1] <= x) ++lo;
    else if (lo > 0 && lam[lo] > x) --lo;
    return lo;
}

}  // namespace

// Shared memory of k_td_fill for a grid of N wavelengths: per segment the cell's Omega_n and
// log-log slope, the segment's integral of Omega lambda, the suffix sums of the integrals of
// Omega, and the grid in FP32.
size_t td_fill_smem_bytes(int N) { return sizeof(double) * 4 * (size_t)N + sizeof(float) * (size_t)N; }

// Spectrum of block b of a launch that starts at spectrum s0: grains in the order `gorder`
// (most bins first), every cell of the chunk for each grain in turn, so that the spectra of one
// launch have similar cost and the largest start first.
__device__ __forceinline__ void td_spectrum(const ChunkDev& ch, const int* gorder, long long s0, int& cell, int& g,
                                            int b = -1) {
    const long long sp = s0 + (b < 0 ? (int)blockIdx.x : b);
    cell = (int)(sp % ch.cells);
    g = gorder[sp / ch.cells];
}

// S blocks per spectrum (cell, grain) of the chunk's cells, each the rows i = part (mod S): q
// [nb][nb] (row-major, rate from row to column) at q + spectrum * qstride, and the absorbed
// power c int Omega on the grid (part 0).
// Downward rates are copied from the grain's table (Dt[u][l], from u to l).  The heating
// rate from i into bin j > i is (1/h) int Omega lambda over the photon wavelengths that end in
// bin j, [hc/(Ehi_j - E_i), hc/(Elo_j - E_i)] (Ehi_M = infinity), plus on j = i + 1 the
// power of the photons too soft to leave bin i, c int_{lambda > hc/(Elo_j - E_i)} Omega,
// over E_j - E_i.  A row's windows tile the grid: each is the closed-form integral of its
// partial end segments plus the segment integrals between them (summed, not differenced);
// the soft term is its partial segment plus a suffix sum.  A warp per row, a lane per j;
// neighbouring lanes share their window edge, and the row ends where the window leaves the
// short-wavelength end of the grid.
__global__ void __launch_bounds__(256) k_td_fill(GrainDev gd, ChunkDev ch, const double* __restrict__ Dt,
                                                 const long long* __restrict__ doff, const int* __restrict__ gorder,
                                                 long long s0, double* q, long long qstride, int S) {
    extern __shared__ double fsm[];
    const int bsp = blockIdx.x / S, part = blockIdx.x % S;  // spectrum of the launch, part of its rows
    int cell, g;
    td_spectrum(ch, gorder, s0, cell, g, bsp);
    const int N = gd.N;
    const double* lam = gd.lam;
    double* om = fsm;
    double* sl = om + N;
    double* I1 = sl + N;
    double* S0 = I1 + N;
    float* l32 = (float*)(S0 + N);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int n = tid; n < N; n += blockDim.x) {
        l32[n] = gd.lam32[n];
        double o = 0.0, sv = 0.0, i0 = 0.0, i1 = 0.0;
        if (n < N - 1) {
            o = ch.ua64[(size_t)n * ch.Cc + cell] * gd.Cact[(size_t)g * N + n];
            sv = ch.su64[(size_t)n * ch.Cc + cell] + gd.sC[(size_t)g * N + n];
            if (o > 0.0) {
                i0 = seg_part(o, sv, lam[n], 0, lam[n], lam[n + 1]);
                i1 = seg_part(o, sv, lam[n], 1, lam[n], lam[n + 1]);
            } else {
                o = 0.0;
            }
        }
        om[n] = o;
        sl[n] = sv;
        I1[n] = i1;
        S0[n] = i0;
    }
    __syncthreads();
    if (warp == 0) {  // suffix sums of the segment integrals of Omega, S0[n] = sum_{m >= n}
        const int per = (N + 31) / 32, b0 = lane * per, b1 = min(N, b0 + per);
        double part = 0.0;
        for (int n = b1 - 1; n >= b0; --n) part += S0[n];
        double above = 0.0;  // sum over the lanes after this one
        for (int o = 1; o < 32; o <<= 1) {
            const double t = __shfl_down_sync(0xffffffffu, part + above, o);
            if (lane + o < 32) above += t;
        }
        for (int n = b1 - 1; n >= b0; --n) {
            above += S0[n];
            S0[n] = above;
        }
    }
    __syncthreads();
    const int off = gd.bin_off[g], nb = gd.bin_off[g + 1] - off;
    const double* E = gd.E + off;
    const double* Dg = Dt + doff[g];
    double* qs = q + (size_t)bsp * qstride;
    const double lam0 = lam[0], lamN = lam[N - 1];
    const int M = nb - 1;
    for (int i = part + S * warp; i < nb; i += S * nw) {
        double* qi = qs + (size_t)i * nb;
        const double* di = Dg + (size_t)i * nb;
        for (int j = lane; j <= i; j += 32) qi[j] = j < i ? di[j] : 0.0;
        const double Ei = E[i];
        int jb = i + 1;
        for (; jb < nb; jb += 32) {
            const int j = jb + lane;
            double lb = 0.0, la = 0.0;
            if (j < nb) lb = kHC / (0.5 * (E[j - 1] + E[j]) - Ei);
            const double nxt = __shfl_down_sync(0xffffffffu, lb, 1);
            if (j < nb) la = j == M ? 0.0 : (lane < 31 ? nxt : kHC / (0.5 * (E[j] + E[j + 1]) - Ei));
            double v = 0.0;
            if (j < nb) {
                const double a = la > lam0 ? la : lam0, b = lb < lamN ? lb : lamN;
                if (b > a) {
                    const int na = seg_of(l32, lam, N, a), nz = seg_of(l32, lam, N, b);
                    if (na == nz) {
                        if (om[na] > 0.0) v = seg_part(om[na], sl[na], lam[na], 1, a, b);
                    } else {
                        if (om[na] > 0.0) v = seg_part(om[na], sl[na], lam[na], 1, a, lam[na + 1]);
                        for (int n = na + 1; n < nz; ++n) v += I1[n];
                        if (om[nz] > 0.0 && b > lam[nz]) v += seg_part(om[nz], sl[nz], lam[nz], 1, lam[nz], b);
                    }
                    v /= kH;
                }
                if (j == i + 1 && lb < lamN) {  // photons too soft to leave bin i
                    const double x = lb > lam0 ? lb : lam0;
                    const int n = seg_of(l32, lam, N, x);
                    double w = S0[n + 1];
                    if (om[n] > 0.0) w += seg_part(om[n], sl[n], lam[n], 0, x, lam[n + 1]);
                    v += kC * w / (E[j] - Ei);
                }
                qi[j] = v;
            }
            if (__all_sync(0xffffffffu, j >= nb || lb <= lam0)) {  // every later window is shortward of the grid
                jb += 32;
                break;
            }
        }
        for (int j = jb + lane; j < nb; j += 32) qi[j] = 0.0;
    }
    if (tid == 0 && part == 0 && ch.pabs) ch.pabs[(size_t)cell * gd.G + g] = kC * S0[0];
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

// Exit rate of state k, s_k = sum_{j < k} q_kj, its reciprocal, and the lowest column with a
// rate out of k (k if none), by one warp; lane 0 stores them.  The lanes read the row as
// j = lane + 32 t, so a warp that has just written the row calls __syncwarp first.
__device__ __forceinline__ void row_exit(const double* qk, int k, double* s, double* rs, int* jlo, int lane) {
    double part = 0.0;
    int jl = k;
    for (int j = lane; j < k; j += 32) {
        const double v = qk[j];
        part += v;
        if (v != 0.0 && j < jl) jl = j;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    jl = __reduce_min_sync(0xffffffffu, jl);
    if (lane == 0) {
        s[k] = part;
        rs[k] = part > 0.0 ? 1.0 / part : 0.0;  // s_k = 0: nothing leaves k downward
        jlo[k] = jl;
    }
}

// One block per spectrum: state reduction of q, back substitution, P and the energy check.
//
// States are removed kGthB at a time (a panel [p0, hi]).  Removing state k adds
// q_ik q_kj / s_k to q_ij for i, j < k.  Inside the panel, step by step, for the rows of the
// panel's remaining states; after the panel, for the rows below it, first their panel columns
// (a sweep over the panel's states in removal order, in registers) and then the block below
// the panel in one pass: sum over the panel's k of q_ik (q_kj / s_k), a rank-kGthB product
// in which q_ik is column k as it stood when k was removed (final from then on: it is the
// column the back substitution reads) and q_kj / s_k is row k at that time, kept in U.  Every
// term stays a sum of products of non-negative numbers; only the order of the additions
// differs from removing the states one by one.  The diagonal of q is never read (s_k sums
// the off-diagonal row), so the updates do not skip it.  The warp that updates the row of the
// next state to be removed also sums it (row_exit), so a step waits on no block-wide sum.
// The fill-in of removing k stays inside the rows that reach k and the columns k reaches:
// rows with no rate into the panel are skipped and columns start at the panel's lowest.
//
// Back substitution, right-looking: X_0 = 1, and once X_i is final every column n > i
// (owned by a fixed thread) takes X_i q_in; X_{i+1} is then complete and its owner divides by
// s_{i+1}.  Past 2^800 every X is scaled by 2^-800 (exact).  P = X / sum X.
//
// SMQ: q is copied into shared memory (row stride nb + 1), for grains of up to kGthSmemBins
// bins; otherwise it is updated in place in device memory, where each panel reads and writes
// the block below it once for kGthB fused multiply-adds per element.
// Shared memory: s, 1/s, X [nb] each, U [kGthB][nb], the lowest columns [nb] (ints, padded
// to doubles), then q (SMQ).
static_assert(kGthB - 1 < kGthThreads / 32, "k_gth: the last warp must be free of panel rows");
template <bool SMQ>
__global__ void __launch_bounds__(kGthThreads, 1) k_gth(GrainDev gd, ChunkDev ch, const int* __restrict__ gorder,
                                                        long long s0, double* q, long long qstride) {
    extern __shared__ double smd[];
    __shared__ double red[kGthThreads / 32];
    __shared__ int rescale;
    int cell, g;
    td_spectrum(ch, gorder, s0, cell, g);
    const int off = gd.bin_off[g], nb = gd.bin_off[g + 1] - off;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kGthThreads / 32;
    double* s = smd;
    double* rs = s + nb;
    double* X = rs + nb;
    double* U = X + nb;
    int* jlo = (int*)(U + kGthB * nb);
    double* qg = q + (size_t)blockIdx.x * qstride;
    double* qs = qg;
    int ld = nb;
    if (SMQ) {
        qs = U + kGthB * nb + (nb + 1) / 2;
        ld = nb + 1;
        for (int i = warp; i < nb; i += nw)
            for (int j = lane; j < nb; j += 32) qs[(size_t)i * ld + j] = qg[(size_t)i * nb + j];
        __syncthreads();
    }
    if (warp == 0) row_exit(qs + (size_t)(nb - 1) * ld, nb - 1, s, rs, jlo, lane);
    if (tid == 0) rescale = 0;
    __syncthreads();
    for (int hi = nb - 1; hi >= 1; hi -= kGthB) {
        const int p0 = hi - kGthB + 1 > 1 ? hi - kGthB + 1 : 1;
        const int nk = hi - p0 + 1;
        for (int k = hi; k >= p0; --k) {
            double* Uk = U + (size_t)(hi - k) * nb;
            const double* qk = qs + (size_t)k * ld;
            const double r = rs[k];
            const int jk = jlo[k];
            // the last warp (never one of the panel's rows below k: at most kGthB - 1 < nw of them)
            // keeps the normalised row for the rows below the panel, while the panel's rows take
            // their multiple of row k directly: no barrier between the two
            if (warp == nw - 1)
                for (int j = lane; j < k; j += 32) Uk[j] = j < jk ? 0.0 : qk[j] * r;
            for (int i = p0 + warp; i < k; i += nw) {  // the panel's rows below k, columns from jk
                double* qi = qs + (size_t)i * ld;
                const double qik = qi[k];
                if (qik != 0.0) {
                    const double c = qik * r;
                    for (int j = jk + lane; j < k; j += 32) qi[j] = fma(c, qk[j], qi[j]);
                }
                if (i == k - 1) {  // the next state to be removed
                    __syncwarp();
                    row_exit(qi, k - 1, s, rs, jlo, lane);
                }
            }
            __syncthreads();
        }
        if (nk > 1)  // rows below the panel: the panel's columns, state by state in removal order
            for (int i = tid; i < p0; i += kGthThreads) {
                double* qi = qs + (size_t)i * ld;
                double x[kGthB];
                bool any = false;
#pragma unroll
                for (int kk = 0; kk < kGthB; ++kk) {
                    const double v = qi[hi - kk > 0 ? hi - kk : 0];
                    x[kk] = kk < nk ? v : 0.0;
                    any |= x[kk] != 0.0;
                }
                if (!any) continue;
#pragma unroll
                for (int kk = 0; kk < kGthB - 1; ++kk) {
                    if (kk < nk - 1 && x[kk] != 0.0) {
                        const double* Uk = U + (size_t)kk * nb;
#pragma unroll
                        for (int k2 = kk + 1; k2 < kGthB; ++k2)
                            if (k2 < nk) x[k2] = fma(x[kk], Uk[hi - k2], x[k2]);
                    }
                }
#pragma unroll
                for (int kk = 1; kk < kGthB; ++kk)
                    if (kk < nk) qi[hi - kk] = x[kk];
            }
        int jp = nb;
        for (int k = p0; k <= hi; ++k) jp = jlo[k] < jp ? jlo[k] : jp;
        __syncthreads();
        // the block below the panel, two rows per warp so that each U value loaded serves both
        // (each element's FMAs in the same order as one row at a time); rows with no rate into
        // the panel are left as they are
        for (int i0 = 2 * warp; i0 < p0; i0 += 2 * nw) {
            const bool has1 = i0 + 1 < p0;
            double* q0 = qs + (size_t)i0 * ld;
            double* q1 = qs + (size_t)(has1 ? i0 + 1 : i0) * ld;
            const double lv0 = lane < nk ? q0[hi - lane] : 0.0;
            const double lv1 = (has1 && lane < nk) ? q1[hi - lane] : 0.0;
            const bool a0 = __ballot_sync(0xffffffffu, lv0 != 0.0) != 0u;
            const bool a1 = __ballot_sync(0xffffffffu, lv1 != 0.0) != 0u;
            if (a0 || a1) {
                double l0[kGthB], l1[kGthB];
#pragma unroll
                for (int kk = 0; kk < kGthB; ++kk) {
                    l0[kk] = __shfl_sync(0xffffffffu, lv0, kk);
                    l1[kk] = __shfl_sync(0xffffffffu, lv1, kk);
                }
                for (int j = jp + lane; j < p0; j += 32) {
                    double v0 = q0[j], v1 = q1[j];
#pragma unroll
                    for (int kk = 0; kk < kGthB; ++kk) {
                        const double u = U[kk * nb + j];
                        v0 = fma(l0[kk], u, v0);
                        v1 = fma(l1[kk], u, v1);
                    }
                    if (a0) q0[j] = v0;
                    if (a1) q1[j] = v1;
                }
            }
            const int inext = p0 - 1;  // the first state of the next panel
            if (inext > 0 && (i0 == inext || (has1 && i0 + 1 == inext))) {
                __syncwarp();
                row_exit(qs + (size_t)inext * ld, inext, s, rs, jlo, lane);
            }
        }
        __syncthreads();
    }
    // back substitution
    for (int n = tid; n < nb; n += kGthThreads) X[n] = n == 0 ? 1.0 : 0.0;
    __syncthreads();
    bool bad = false;
    for (int i = 0; i + 1 < nb; ++i) {
        const double xi = X[i];
        const double* qi = qs + (size_t)i * ld;
        for (int n = tid; n < nb; n += kGthThreads) {
            if (n <= i) continue;
            double a = fma(xi, qi[n], X[n]);
            if (n == i + 1) {  // every state below n has contributed
                if (s[n] == 0.0) {
                    bad |= a != 0.0;
                    a = 0.0;
                } else {
                    a *= rs[n];
                }
                if (a > 0x1p800) rescale = 1;
            }
            X[n] = a;
        }
        __syncthreads();
        if (rescale) {
            for (int n = tid; n < nb; n += kGthThreads) X[n] *= 0x1p-800;
            __syncthreads();
            if (tid == 0) rescale = 0;
            __syncthreads();
        }
    }
    bad = __syncthreads_or(bad);
    double part = 0.0;
    for (int i = tid; i < nb; i += kGthThreads) part += X[i];
    const double inv = 1.0 / block_sum(part, red);
    double emit = 0.0;
    double* prow = ch.P + (size_t)cell * ch.ldP + off;
    for (int i = tid; i < nb; i += kGthThreads) {
        const double p = X[i] * inv;
        prow[i] = p;
        emit = fma(p, gd.cde[off + i], emit);
    }
    emit = block_sum(emit, red);
    if (tid == 0) {
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

size_t gth_smem_bytes(int max_bins) {
    const size_t vec = sizeof(double) * ((size_t)(3 + kGthB) * max_bins + (max_bins + 1) / 2);
    return max_bins <= kGthSmemBins ? vec + sizeof(double) * (size_t)max_bins * (max_bins + 1) : vec;
}

long long discrete_batch_spectra(const GrainDev& g, const ChunkDev& ch, long long s0, long long batch) {
    const long long spectra = (long long)ch.cells * g.G;
    return spectra - s0 < batch ? spectra - s0 : batch;
}

cudaError_t launch_discrete_fill(const GrainDev& g, const ChunkDev& ch, const double* D, const long long* doff,
                                 const int* gorder, double* q, long long qstride, long long s0, long long n,
                                 cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = td_fill_smem_bytes(g.N);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_td_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    // parts per spectrum (rows by residue): about two blocks per SM when the launch has few spectra
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int S = (int)(n >= 2LL * sms ? 1 : std::min(16LL, std::max(1LL, 2LL * sms / n)));
    k_td_fill<<<(unsigned)(n * S), 256, smem, st>>>(g, ch, D, doff, gorder, s0, q, qstride, S);
    return cudaGetLastError();
}

cudaError_t launch_discrete_gth(const GrainDev& g, const ChunkDev& ch, const int* gorder, double* q, long long qstride,
                                long long s0, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const bool smq = g.max_bins <= kGthSmemBins;
    const size_t smem = gth_smem_bytes(g.max_bins);
    if (smem > 48 * 1024) {
        cudaError_t e = smq ? cudaFuncSetAttribute(k_gth<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                            : cudaFuncSetAttribute(k_gth<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (smq)
        k_gth<true><<<(unsigned)n, kGthThreads, smem, st>>>(g, ch, gorder, s0, q, qstride);
    else
        k_gth<false><<<(unsigned)n, kGthThreads, smem, st>>>(g, ch, gorder, s0, q, qstride);
    return cudaGetLastError();
}

}  // namespace heat
