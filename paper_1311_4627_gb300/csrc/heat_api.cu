// Host side of libheat: context, grain set-up (band and pattern tables), field
// staging, chunked solve and the C ABI declared in include/heat.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/heat.h"
#include "common.cuh"
#include "ctx.h"
#include "emis_tc.h"
#include "internal.h"

using namespace heat;

// launch `call` on stream st, bracketed by timing events when o.timing is set
#define TIMED(kind, call)                                  \
    do {                                                   \
        cudaEvent_t ea_ = nullptr, eb_ = nullptr;          \
        if (o.timing) {                                    \
            ea_ = ctx->take_event();                       \
            CKR(cudaEventRecord(ea_, cs));                 \
        }                                                  \
        CKR(call);                                         \
        if (o.timing) {                                    \
            eb_ = ctx->take_event();                       \
            CKR(cudaEventRecord(eb_, cs));                 \
            ctx->timed.push_back({(kind), ea_, eb_});      \
        }                                                  \
    } while (0)

#define CKR(call)                                         \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return ctx->cuda_fail(e_, #call); \
    } while (0)

namespace {

const double kHChost = 6.62607015e-27 * 2.99792458e10;
const double kHhost = 6.62607015e-27;
const double kChost = 2.99792458e10;

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// largest n in [0, N-2] with lam[n] <= x (x inside the grid)
int segment_of(const std::vector<double>& lam, double x) {
    int lo = 0, hi = (int)lam.size() - 2;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (lam[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename T>
cudaError_t upload(DevBuf& b, const std::vector<T>& v) {
    size_t bytes = std::max<size_t>(v.size() * sizeof(T), 16);
    cudaError_t e = b.ensure(bytes);
    if (e != cudaSuccess) return e;
    if (v.empty()) return cudaSuccess;
    return cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    }
    return fn;
}

// 2D K-major operand map: rows x kp elements, 128-byte swizzle, box = (128-byte slice, box_rows).
bool encode_operand(CUtensorMap* m, void* base, bool tf32, long long kp, long long rows, int box_rows) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    size_t es = tf32 ? 4 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(kp * es)};
    cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool mode_tf32(int m) { return m == HEAT_EMIS_TF32X3 || m == HEAT_EMIS_TF32; }
bool mode_split(int m) { return m == HEAT_EMIS_BF16X3 || m == HEAT_EMIS_TF32X3; }

}  // namespace

// Build the B' operands and column scales of a tensor-core mode (once per mode).  Per-grain
// output: one operand per grain from K_g.  Size-integrated output (si): a single operand over
// all bins of all grains from the size-weighted kernel Kw, so that one GEMM with K = sum of
// the grains' bins accumulates sum_g w_g j_g in the tensor memory.
static heat_status ensure_tc_mode(heat_ctx* ctx, int m, bool si, cudaStream_t st) {
    auto& t = si ? ctx->tc_si[m] : ctx->tc[m];
    if (t.built) return HEAT_OK;
    const int G = si ? 1 : ctx->G, N = ctx->N;
    const bool tf32 = mode_tf32(m), split = mode_split(m);
    const int ke = tf32 ? 32 : 64;
    t.kp_h.resize(G);
    t.boff_h.resize(G + 1);
    t.boff_h[0] = 0;
    for (int g = 0; g < G; ++g) {
        int nb = si ? ctx->nbt : ctx->bin_off[g + 1] - ctx->bin_off[g];
        t.kp_h[g] = (split ? 2 : 1) * ((nb + ke - 1) / ke * ke);  // [hi | lo] parts of whole k blocks
        t.boff_h[g + 1] = t.boff_h[g] + (long long)N * t.kp_h[g];
    }
    t.order.resize(G);
    for (int g = 0; g < G; ++g) t.order[g] = g;
    std::stable_sort(t.order.begin(), t.order.end(), [&](int a, int b) { return t.kp_h[a] > t.kp_h[b]; });
    size_t es = tf32 ? 4 : 2;
    if (t.B.ensure(es * (size_t)t.boff_h[G]) || t.colscale.ensure(sizeof(float) * (size_t)G * N) ||
        upload(t.kp, t.kp_h) || upload(t.boff, t.boff_h))
        return ctx->fail(HEAT_ENOMEM, "heat_solve: allocation of tensor-core operands failed");
    CKR(launch_pack_k(N, G, si ? ctx->d_koff_all.as<int>() : ctx->d_bin_off.as<int>(),
                      si ? ctx->d_Kw.as<double>() : ctx->d_K.as<double>(), t.boff.as<long long>(), t.kp.as<int>(),
                      split, tf32, t.B.p, t.colscale.as<float>(), st));
    t.built = true;
    return HEAT_OK;
}

// Row offsets of the packed P operands for chunks of Cc_alloc cells (uploaded once per
// chunk size, before any chunk is launched).
static heat_status prepare_tc_rows(heat_ctx* ctx, int m, bool si, int Cc_alloc) {
    auto& t = si ? ctx->tc_si[m] : ctx->tc[m];
    if (t.aoff_cells == Cc_alloc) return HEAT_OK;
    const int G = si ? 1 : ctx->G;
    t.aoff_h.assign(G + 1, 0);
    for (int g = 0; g < G; ++g) t.aoff_h[g + 1] = t.aoff_h[g] + (long long)Cc_alloc * t.kp_h[g];
    CKR(cudaDeviceSynchronize());  // earlier solves may still read the old offsets
    if (upload(t.aoff, t.aoff_h)) return ctx->fail(HEAT_ENOMEM, "heat_solve: allocation failed");
    t.aoff_cells = Cc_alloc;
    return HEAT_OK;
}

// Tensor-core emissivity of one chunk whose P rows are ready at P (row stride nbt), or, with
// `packed`, whose operand A' and row scales the recursion has written: per-grain j
// [cells][G][N], or with si the size-integrated J [cells][N].  A / rowscale: the slot's
// operand buffers (sized by the caller).
static heat_status emis_tc_chunk(heat_ctx* ctx, int m, bool si, const double* P, int cells, void* A, float* rowscale,
                                 void* jdst, bool j_f64, bool packed, int ntile, cudaStream_t st) {
    auto& t = si ? ctx->tc_si[m] : ctx->tc[m];
    const int G = si ? 1 : ctx->G, N = ctx->N;
    const bool tf32 = mode_tf32(m), split = mode_split(m);
    const size_t es = tf32 ? 4 : 2;
    if (!packed)  // else the recursion's epilogue has written A' and the row scales
        CKR(launch_pack_p(cells, G, si ? ctx->d_koff_all.as<int>() : ctx->d_bin_off.as<int>(), P, ctx->nbt,
                          t.aoff.as<long long>(), t.kp.as<int>(), split, tf32, A, rowscale, st));
    EmisTcParams prm;  // ~25 KB of tensor maps, copied into the launch's parameters
    for (int g0 = 0; g0 < G; g0 += kMaxTcGrains) {
        int ng = std::min(kMaxTcGrains, G - g0);
        std::memset(&prm, 0, sizeof(prm));
        for (int i = 0; i < ng; ++i) {
            int g = t.order[g0 + i];
            char* abase = (char*)A + es * (size_t)t.aoff_h[g];
            char* bbase = (char*)t.B.p + es * (size_t)t.boff_h[g];
            if (!encode_operand(&prm.ta[i], abase, tf32, t.kp_h[g], cells, 128) ||
                !encode_operand(&prm.tb[i], bbase, tf32, t.kp_h[g], N, ntile))
                return ctx->fail(HEAT_ECUDA, "heat_solve: cuTensorMapEncodeTiled failed");
            prm.ksteps[i] = (split ? t.kp_h[g] / 2 : t.kp_h[g]) / (tf32 ? 32 : 64);
            prm.grain[i] = g;
        }
        prm.ng = ng;
        prm.cells = cells;
        prm.N = N;
        prm.G = G;
        prm.mtiles = (cells + 127) / 128;
        prm.ntiles = (N + ntile - 1) / ntile;
        prm.rowscale = rowscale;
        prm.colscale = t.colscale.as<float>();
        prm.j = jdst;
        prm.ldj = (long long)G * N;
        prm.j_f64 = j_f64 ? 1 : 0;
        prm.status = ctx->d_status.as<int>();
        prm.wait_polls = ctx->wait_polls;
        CKR(launch_emis_tc(prm, tf32, split, ntile, ctx->sms, st));
    }
    return HEAT_OK;
}

// Grain orders, longest first: the recursion's by band + row_weight x rows (a long chain of
// narrow rows takes its time whatever the load, so it starts early; heat_autotune can pick the
// weight), the build's by band + 12 x rows.
static void order_grains(heat_ctx* ctx) {
    const int G = ctx->G;
    std::vector<long long> cost(G), cost_build(G);
    for (int g = 0; g < G; ++g) {
        cost[g] = ctx->grain_band[g] + (long long)ctx->row_weight * ctx->grain_rows[g];
        cost_build[g] = ctx->grain_band[g] + 12LL * ctx->grain_rows[g];
    }
    ctx->grain_order.resize(G);
    ctx->grain_order_build.resize(G);
    for (int g = 0; g < G; ++g) ctx->grain_order[g] = ctx->grain_order_build[g] = g;
    std::stable_sort(ctx->grain_order.begin(), ctx->grain_order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::stable_sort(ctx->grain_order_build.begin(), ctx->grain_order_build.end(),
                     [&](int a, int b) { return cost_build[a] > cost_build[b]; });
    ctx->tasks_NG = -1;  // the task lists follow the orders
    ctx->tail_NG = -1;
}

// (grain, group) task lists of a chunk of NG groups: the recursion's order, then the build's.
static std::vector<int2> make_tasks(const heat_ctx* ctx, int NG) {
    std::vector<int2> tasks;
    tasks.reserve(2 * (size_t)ctx->G * NG);
    // recursion: near-chain grains (fewer than 8 band elements per row: their time is the
    // per-row latency, they hardly use the FP64 unit) interleaved with the wide-band grains
    // in proportion to each list's cost, so that every SM holds both kinds throughout
    std::vector<int> chain, wide;
    for (int g : ctx->grain_order) (ctx->grain_band[g] < 8LL * ctx->grain_rows[g] ? chain : wide).push_back(g);
    auto cost = [&](int g) { return (double)(ctx->grain_band[g] + (long long)ctx->row_weight * ctx->grain_rows[g]); };
    double tc = 0.0, tw = 0.0, dc = 0.0, dw = 0.0;
    for (int g : chain) tc += cost(g);
    for (int g : wide) tw += cost(g);
    size_t ic = 0, iw = 0;
    while (ic < chain.size() || iw < wide.size()) {
        const bool take_chain = iw == wide.size() || (ic < chain.size() && dc / tc <= dw / tw);
        const int g = take_chain ? chain[ic++] : wide[iw++];
        (take_chain ? dc : dw) += cost(g);
        for (int grp = 0; grp < NG; ++grp) tasks.push_back(make_int2(g, grp));
    }
    for (int gi = 0; gi < ctx->G; ++gi)
        for (int grp = 0; grp < NG; ++grp) tasks.push_back(make_int2(ctx->grain_order_build[gi], grp));
    return tasks;
}

extern "C" {

void heat_default_opts(heat_opts* o) {
    if (!o) return;
    o->build = HEAT_BUILD_F64;
    o->emis = HEAT_EMIS_F64;
    o->j_dtype = HEAT_F64;
    o->size_integrate = 0;
    o->cell_begin = 0;
    o->cell_count = 0;
    o->chunk_cells = 0;
    o->host_io = 0;
    o->timing = 0;
    o->ledger_out = nullptr;
    o->streams = 0;
    o->heating = HEAT_HEATING_INTEGRAL;
    o->prune_eps = 0.0;
    o->fused_build = 0;
    o->recur_blocks_per_sm = 0;
    o->emis_n_tile = 0;
    o->build_prefetch = 0;
    o->cooling = HEAT_COOLING_CONTINUOUS;
}

heat_status heat_create_grid(heat_ctx** out, int device, int n_lambda, const double* lambda_cm) {
    if (!out) return HEAT_EINVAL;
    *out = nullptr;
    if (n_lambda < 2 || !lambda_cm) return HEAT_EINVAL;
    for (int n = 0; n < n_lambda; ++n) {
        if (!(lambda_cm[n] > 0.0) || !std::isfinite(lambda_cm[n])) return HEAT_EINVAL;
        if (n > 0 && !(lambda_cm[n] > lambda_cm[n - 1])) return HEAT_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return HEAT_ECUDA;
    heat_ctx* ctx = new (std::nothrow) heat_ctx();
    if (!ctx) return HEAT_ENOMEM;
    ctx->device = device;
    ctx->N = n_lambda;
    ctx->lam.assign(lambda_cm, lambda_cm + n_lambda);
    auto cleanup = [&](heat_status s) { heat_destroy(ctx); return s; };
    if (cudaSetDevice(device) != cudaSuccess) return cleanup(HEAT_ECUDA);
    std::vector<double> dln(n_lambda - 1);
    std::vector<float> lam32(n_lambda), dln32(n_lambda - 1);
    for (int n = 0; n < n_lambda - 1; ++n) {
        dln[n] = std::log(lambda_cm[n + 1] / lambda_cm[n]);
        dln32[n] = (float)dln[n];
    }
    for (int n = 0; n < n_lambda; ++n) lam32[n] = (float)lambda_cm[n];
    if (upload(ctx->d_lam, ctx->lam) != cudaSuccess || upload(ctx->d_dln, dln) != cudaSuccess ||
        upload(ctx->d_lam32, lam32) != cudaSuccess || upload(ctx->d_dln32, dln32) != cudaSuccess)
        return cleanup(HEAT_ENOMEM);
    if (ctx->d_status.ensure(sizeof(int)) != cudaSuccess) return cleanup(HEAT_ENOMEM);
    if (cudaMemset(ctx->d_status.p, 0, sizeof(int)) != cudaSuccess) return cleanup(HEAT_ECUDA);
    if (cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return cleanup(HEAT_ECUDA);
    double glx[kGLPoints], glw[kGLPoints];
    gauss_legendre(kGLPoints, glx, glw);
    if (set_gauss_legendre(glx, glw) != cudaSuccess) return cleanup(HEAT_ECUDA);
    {
        std::vector<double> gl(glx, glx + kGLPoints);
        gl.insert(gl.end(), glw, glw + kGLPoints);
        if (upload(ctx->d_gl, gl) != cudaSuccess) return cleanup(HEAT_ENOMEM);
    }
    *out = ctx;
    return HEAT_OK;
}

heat_status heat_set_grains(heat_ctx* ctx, int n_grains, const double* radius_cm, const double* c_abs_cm2,
                            const int* bin_offset, const double* T_bins_K, const double* H_bins_erg,
                            const double* size_weight) {
    if (!ctx) return HEAT_EINVAL;
    if (n_grains < 1 || !radius_cm || !c_abs_cm2 || !bin_offset || !T_bins_K || !H_bins_erg)
        return ctx->fail(HEAT_EINVAL, "heat_set_grains: null argument or n_grains < 1");
    const int N = ctx->N, G = n_grains;
    if (bin_offset[0] != 0) return ctx->fail(HEAT_EINVAL, "heat_set_grains: bin_offset[0] must be 0");
    for (int g = 0; g < G; ++g) {
        int nb = bin_offset[g + 1] - bin_offset[g];
        if (nb < 2 || nb > 4096) return ctx->fail(HEAT_EINVAL, "heat_set_grains: each grain needs 2..4096 bins");
        if (!(radius_cm[g] > 0.0)) return ctx->fail(HEAT_EINVAL, "heat_set_grains: radius must be > 0");
        for (int n = 0; n < N; ++n) {
            double c = c_abs_cm2[(size_t)g * N + n];
            if (!(c >= 0.0) || !std::isfinite(c)) return ctx->fail(HEAT_EINVAL, "heat_set_grains: bad C_abs");
        }
        for (int i = bin_offset[g]; i < bin_offset[g + 1]; ++i) {
            if (!(T_bins_K[i] > 0.0) || !(H_bins_erg[i] > 0.0) || !std::isfinite(T_bins_K[i]) ||
                !std::isfinite(H_bins_erg[i]))
                return ctx->fail(HEAT_EINVAL, "heat_set_grains: T and H must be positive and finite");
            if (i > bin_offset[g] && !(T_bins_K[i] > T_bins_K[i - 1] && H_bins_erg[i] > H_bins_erg[i - 1]))
                return ctx->fail(HEAT_EINVAL, "heat_set_grains: T and H must ascend within a grain");
        }
    }
    if (size_weight)
        for (int g = 0; g < G; ++g)
            if (!std::isfinite(size_weight[g])) return ctx->fail(HEAT_EINVAL, "heat_set_grains: bad size weight");
    CKR(cudaSetDevice(ctx->device));
    const int nbt = bin_offset[G];
    const std::vector<double>& lam = ctx->lam;
    ctx->G = G;
    ctx->nbt = nbt;
    ctx->bin_off.assign(bin_offset, bin_offset + G + 1);
    ctx->radius.assign(radius_cm, radius_cm + G);
    ctx->has_w = size_weight != nullptr;
    ctx->w.assign(G, 0.0);
    if (size_weight) std::copy(size_weight, size_weight + G, ctx->w.begin());
    ctx->tasks_NG = -1;
    ctx->tail_NG = -1;
    ctx->tuned_streams = ctx->tuned_chunk = 0;
    ctx->tuned_prefetch = 0;
    ctx->row_weight = 30;
    ctx->td_built = false;
    for (auto* modes : {ctx->tc, ctx->tc_si})
        for (int m = 0; m < 5; ++m) {
            modes[m].built = false;
            modes[m].aoff_cells = -1;
        }

    // per-grain cross-section tables
    std::vector<double> Cact((size_t)G * N, 0.0), sC((size_t)G * N, 0.0);
    std::vector<float> ca32((size_t)G * N, 0.0f), ce32((size_t)G * N, 0.0f), sC32((size_t)G * N, 0.0f);
    for (int g = 0; g < G; ++g) {
        const double* C = c_abs_cm2 + (size_t)g * N;
        for (int n = 0; n < N - 1; ++n) {
            if (C[n] > 0.0 && C[n + 1] > 0.0) {
                size_t k = (size_t)g * N + n;
                Cact[k] = C[n];
                sC[k] = std::log(C[n + 1] / C[n]) / std::log(lam[n + 1] / lam[n]);
                ca32[k] = (float)(C[n] * lam[n] * lam[n] / kHhost);
                ce32[k] = (float)(kChost * C[n] * lam[n]);
                sC32[k] = (float)sC[k];
            }
        }
    }
    // bins, band and soft-photon tables
    std::vector<double> invdE(nbt, 0.0);
    std::vector<float> invdE32(nbt, 0.0f);
    std::vector<int> rowptr;
    rowptr.reserve(nbt + G);
    std::vector<PatF64> pat64;
    std::vector<PatF32> pat32;
    std::vector<int> seg_ptr((size_t)G * (N + 1), 0);
    std::vector<SoftF64> soft;
    std::vector<int> soft_off(G + 1, 0);
    std::vector<int> wmax(G, 1);
    std::vector<int> bin_grain(nbt);
    ctx->grain_band.assign(G, 0);
    ctx->grain_rows.assign(G, 0);
    long long band_total = 0;
    struct Ent {
        int n, e;
        double t;
    };
    std::vector<int> diag_e(nbt, 0), diag_ok(nbt, 0);
    std::vector<PointEnt> pent;  // point-rule entries (Eq. heating), column by column
    std::vector<RowEnt32> rent;  // every band element in row order (fused kernel)
    std::vector<int> pcol(nbt + 1, 0);
    for (int g = 0; g < G; ++g) {
        const int off = bin_offset[g], nb = bin_offset[g + 1] - off, M = nb - 1;
        const double* E = H_bins_erg + off;
        std::vector<double> Elo(nb);
        Elo[0] = 0.0;
        for (int i = 1; i < nb; ++i) Elo[i] = 0.5 * (E[i - 1] + E[i]);
        for (int i = 0; i < nb; ++i) bin_grain[off + i] = g;
        for (int j = 0; j < M; ++j) {
            invdE[off + j] = 1.0 / (E[j + 1] - E[j]);
            invdE32[off + j] = (float)invdE[off + j];
        }
        long long band = 0;
        std::vector<Ent> ents;
        std::vector<int> row_e(nb, 0), row_jlo(nb, 0);  // band index of (f, jlo(f)) and jlo(f)
        // row 0 has no elements
        rowptr.push_back((int)band_total);
        for (int f = 1; f <= M; ++f) {
            rowptr.push_back((int)(band_total + band));
            int jlo = f;
            for (int j = f - 1; j >= 0; --j) {
                if (kHChost / (Elo[f] - E[j]) < lam[0]) break;
                jlo = j;
            }
            // the diagonal element (f, f-1) is always stored: it carries the intra-bin
            // term even when no photon on the grid reaches bin f from bin f-1
            const bool diag_in_band = jlo < f;
            if (!diag_in_band) jlo = f - 1;
            row_e[f] = (int)(band_total + band);
            row_jlo[f] = jlo;
            if (f > 1 && jlo < row_jlo[f - 1])  // the recursion kernels rely on band starts never decreasing
                return ctx->fail(HEAT_EINVAL, "heat_set_grains: band starts decrease (non-monotonic enthalpies?)");
            wmax[g] = std::max(wmax[g], f - jlo);
            diag_e[off + f - 1] = (int)(band_total + band + (f - 1 - jlo));
            diag_ok[off + f - 1] = diag_in_band ? 1 : 0;
            for (int j = jlo; j < f; ++j) {
                double lf = kHChost / (Elo[f] - E[j]);
                Ent en;
                en.e = (int)(band_total + band);
                RowEnt32 re;
                re.n = N;  // no photon part unless the pattern loop below sets the segment
                re.t = re.cat = re.zt = 0.0f;
                rent.push_back(re);
                if (!diag_in_band) {  // below the grid: no photon part, no pattern entry
                    ++band;
                    continue;
                }
                if (lf >= lam[N - 1]) {
                    en.n = N - 1;
                    en.t = 0.0;
                } else {
                    en.n = segment_of(lam, lf);
                    en.t = std::log(lf / lam[en.n]);
                }
                ents.push_back(en);
                ++band;
            }
        }
        rowptr.push_back((int)(band_total + band));
        // point-rule entries: column j holds rows j+1 .. F(j), a contiguous range since
        // jlo(f) does not decrease with f; every element the point rule can make non-zero
        // (E_u - E_j <= hc/lambda_0) lies in the band, and the band's other elements take the
        // column's suffix sum with T = 0
        for (int j = 0; j < nb; ++j) {
            pcol[off + j] = (int)pent.size();
            int F = j;
            while (F + 1 <= M && row_jlo[F + 1] <= j) ++F;
            for (int u = F; u > j; --u) {
                PointEnt pe;
                pe.e = row_e[u] + (j - row_jlo[u]);
                const double x = kHChost / (E[u] - E[j]);
                const double dE = u < M ? Elo[u + 1] - Elo[u] : E[M] - E[M - 1];  // upper bin's width
                if (x >= lam[0] && x <= lam[N - 1]) {
                    pe.n = segment_of(lam, x);
                    pe.t = std::log(x / lam[pe.n]);
                    pe.fac = x * x * x * dE / (kHhost * kHhost * kChost);
                } else {
                    pe.n = -1;
                    pe.t = 0.0;
                    pe.fac = 0.0;
                }
                pent.push_back(pe);
            }
        }
        // pattern: the grain's elements grouped by segment
        std::stable_sort(ents.begin(), ents.end(), [](const Ent& a, const Ent& b) { return a.n < b.n; });
        size_t base = pat64.size();
        size_t k = 0;
        for (int n = 0; n <= N; ++n) {
            while (k < ents.size() && ents[k].n < n) ++k;
            seg_ptr[(size_t)g * (N + 1) + n] = (int)(base + k);
        }
        for (const Ent& en : ents) {
            size_t kk = (size_t)g * N + en.n;
            double ca = (en.n < N - 1) ? Cact[kk] * lam[en.n] * lam[en.n] / kHhost : 0.0;
            double s2 = (en.n < N - 1) ? sC[kk] + 2.0 : 0.0;
            PatF64 a;
            a.e = en.e;
            a.pad = en.n;
            a.t = en.t;
            PatF32 b;
            b.e = en.e;
            b.t = (float)en.t;
            b.cat = (float)(ca * en.t);
            b.zt = (float)(s2 * en.t);
            pat64.push_back(a);
            pat32.push_back(b);
            RowEnt32& re = rent[(size_t)en.e];  // the same element in row order
            re.n = en.n;
            re.t = b.t;
            re.cat = b.cat;
            re.zt = b.zt;
        }
        // soft-photon abscissae, sorted by segment, descending
        soft_off[g] = (int)soft.size();
        std::vector<SoftF64> sg;
        for (int j = 0; j < M; ++j) {
            double ls = kHChost / (Elo[j + 1] - E[j]);
            SoftF64 sf;
            sf.j = j;
            sf.e_diag = diag_e[off + j];
            sf.diag_in_band = diag_ok[off + j];
            if (ls < lam[0]) {
                sf.n = -1;
                sf.t = 0.0;
            } else if (ls >= lam[N - 1]) {
                sf.n = N - 1;
                sf.t = 0.0;
            } else {
                sf.n = segment_of(lam, ls);
                sf.t = std::log(ls / lam[sf.n]);
            }
            sg.push_back(sf);
        }
        std::stable_sort(sg.begin(), sg.end(), [](const SoftF64& a, const SoftF64& b) { return a.n > b.n; });
        soft.insert(soft.end(), sg.begin(), sg.end());
        band_total += band;
        if (band_total * 32 >= 0x7fffffffLL)
            return ctx->fail(HEAT_EINVAL, "heat_set_grains: band of the grains too large (over 6.7e7 elements)");
        // task order (longest first): a row costs about as much as 12 band elements in
        // the recursion (its chain waits on dependent FP64 ops), so many-row grains start early
        ctx->grain_band[g] = band;
        ctx->grain_rows[g] = nb;
    }
    soft_off[G] = (int)soft.size();
    pcol[nbt] = (int)pent.size();
    if ((long long)pent.size() != band_total || (long long)rent.size() != band_total)
        return ctx->fail(HEAT_EINVAL, "heat_set_grains: element tables do not cover the band");
    {   // padding: the fused kernel makes its B values in whole runs that may pass the end
        RowEnt32 pad;
        pad.n = N;
        pad.t = pad.cat = pad.zt = 0.0f;
        rent.insert(rent.end(), 128, pad);
    }
    pat32.resize(pat32.size() + 64, PatF32{});  // the FP32 build prefetches 32 entries past a segment's end
    ctx->band_per_cell = band_total;
    ctx->band_max = 0;
    ctx->wmax_all = *std::max_element(wmax.begin(), wmax.end());
    for (int g = 0; g < G; ++g) ctx->band_max = std::max(ctx->band_max, (int)ctx->grain_band[g]);
    ctx->max_bins = 0;
    for (int g = 0; g < G; ++g) ctx->max_bins = std::max(ctx->max_bins, bin_offset[g + 1] - bin_offset[g]);
    order_grains(ctx);

    std::vector<double> cabs(c_abs_cm2, c_abs_cm2 + (size_t)G * N), T(T_bins_K, T_bins_K + nbt),
        E(H_bins_erg, H_bins_erg + nbt);
    std::vector<int> boff(bin_offset, bin_offset + G + 1);
    if (upload(ctx->d_bin_off, boff) || upload(ctx->d_cabs, cabs) || upload(ctx->d_T, T) || upload(ctx->d_E, E) ||
        upload(ctx->d_invdE, invdE) || upload(ctx->d_invdE32, invdE32) || upload(ctx->d_Cact, Cact) ||
        upload(ctx->d_sC, sC) || upload(ctx->d_ca32, ca32) || upload(ctx->d_ce32, ce32) ||
        upload(ctx->d_sC32, sC32) || upload(ctx->d_rowptr, rowptr) || upload(ctx->d_wmax, wmax) || upload(ctx->d_pat64, pat64) ||
        upload(ctx->d_pat32, pat32) || upload(ctx->d_seg_ptr, seg_ptr) || upload(ctx->d_soft, soft) || upload(ctx->d_soft_off, soft_off) ||
        upload(ctx->d_w, ctx->w) || upload(ctx->d_pent, pent) || upload(ctx->d_pcol, pcol) ||
        upload(ctx->d_rent, rent))
        return ctx->fail(HEAT_ENOMEM, "heat_set_grains: device allocation failed");
    std::vector<int> koff_all = {0, nbt};
    if (upload(ctx->d_koff_all, koff_all)) return ctx->fail(HEAT_ENOMEM, "heat_set_grains: device allocation failed");

    // cooling rates on the device
    std::vector<int2> work;
    for (int g = 0; g < G; ++g)
        for (int f = 1; f < bin_offset[g + 1] - bin_offset[g]; ++f) work.push_back(make_int2(g, f));
    DevBuf d_work, d_bg;
    if (upload(d_work, work) || upload(d_bg, bin_grain))
        return ctx->fail(HEAT_ENOMEM, "heat_set_grains: device allocation failed");
    if (ctx->d_Cf.ensure(sizeof(double) * nbt)) return ctx->fail(HEAT_ENOMEM, "heat_set_grains: allocation");
    CKR(cudaMemset(ctx->d_Cf.p, 0, sizeof(double) * nbt));
    CKR(launch_cooling(N, ctx->d_lam.as<double>(), ctx->d_cabs.as<double>(), ctx->d_bin_off.as<int>(), G,
                       ctx->d_T.as<double>(), ctx->d_E.as<double>(), ctx->d_Cf.as<double>(), d_work.as<int2>(),
                       (int)work.size(), 0));
    size_t kbytes = sizeof(double) * (size_t)nbt * N;
    if (ctx->d_K.ensure(kbytes)) return ctx->fail(HEAT_ENOMEM, "heat_set_grains: allocation of Planck kernels");
    if (ctx->has_w && ctx->d_Kw.ensure(kbytes))
        return ctx->fail(HEAT_ENOMEM, "heat_set_grains: allocation of Planck kernels");
    CKR(launch_planck(N, nbt, ctx->d_lam.as<double>(), ctx->d_cabs.as<double>(), d_bg.as<int>(), ctx->d_T.as<double>(),
                      ctx->d_E.as<double>(), ctx->d_w.as<double>(), ctx->d_K.as<double>(),
                      ctx->has_w ? ctx->d_Kw.as<double>() : nullptr, 0));
    if (ctx->d_kexp.ensure(sizeof(int) * nbt)) return ctx->fail(HEAT_ENOMEM, "heat_set_grains: allocation");
    CKR(launch_kexp(N, nbt, ctx->d_K.as<double>(), ctx->d_kexp.as<int>(), 0));
    CKR(cudaDeviceSynchronize());
    std::vector<double> Cf(nbt), invC(nbt, 0.0), cde(nbt, 0.0);
    CKR(cudaMemcpy(Cf.data(), ctx->d_Cf.p, sizeof(double) * nbt, cudaMemcpyDeviceToHost));
    for (int g = 0; g < G; ++g)
        for (int i = bin_offset[g] + 1; i < bin_offset[g + 1]; ++i) {
            invC[i] = Cf[i] > 0.0 ? 1.0 / Cf[i] : 0.0;
            cde[i] = Cf[i] * (H_bins_erg[i] - H_bins_erg[i - 1]);
        }
    if (upload(ctx->d_invC, invC) || upload(ctx->d_cde, cde))
        return ctx->fail(HEAT_ENOMEM, "heat_set_grains: allocation");
    d_work.release();
    d_bg.release();
    return HEAT_OK;
}

heat_status heat_set_fields(heat_ctx* ctx, int n_cells, const void* u, int dtype, int on_device, void* stream) {
    if (!ctx) return HEAT_EINVAL;
    if (n_cells < 0 || (n_cells > 0 && !u) || (dtype != HEAT_F64 && dtype != HEAT_F32))
        return ctx->fail(HEAT_EINVAL, "heat_set_fields: bad argument");
    CKR(cudaSetDevice(ctx->device));
    ctx->n_cells = n_cells;
    ctx->u_dtype = dtype;
    if (on_device) {
        ctx->u_dev = u;
        return HEAT_OK;
    }
    size_t bytes = (size_t)n_cells * ctx->N * (dtype == HEAT_F64 ? 8 : 4);
    if (ctx->d_u_own.ensure(std::max<size_t>(bytes, 16)))
        return ctx->fail(HEAT_ENOMEM, "heat_set_fields: device allocation failed");
    if (bytes) CKR(cudaMemcpyAsync(ctx->d_u_own.p, u, bytes, cudaMemcpyHostToDevice, (cudaStream_t)stream));
    ctx->u_dev = ctx->d_u_own.p;
    return HEAT_OK;
}

// Thermal-discrete downward rates of every grain (once per grain set, on first use).
static heat_status ensure_discrete(heat_ctx* ctx, cudaStream_t st) {
    if (ctx->td_built) return HEAT_OK;
    const int G = ctx->G;
    std::vector<long long> doff(G + 1, 0), woff(G + 1, 0);
    for (int g = 0; g < G; ++g) {
        const long long nb = ctx->bin_off[g + 1] - ctx->bin_off[g];
        doff[g + 1] = doff[g] + nb * nb;
        woff[g + 1] = woff[g] + nb * (nb - 1) / 2;
    }
    std::vector<int> order(G);  // grains with the most bins first (the solve's launch order)
    for (int g = 0; g < G; ++g) order[g] = g;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return ctx->bin_off[a + 1] - ctx->bin_off[a] > ctx->bin_off[b + 1] - ctx->bin_off[b];
    });
    if (ctx->d_Dtd.ensure(sizeof(double) * (size_t)std::max(1LL, doff[G])) || upload(ctx->d_Dtd_off, doff) ||
        upload(ctx->d_Dtd_woff, woff) || upload(ctx->d_Dtd_order, order))
        return ctx->fail(HEAT_ENOMEM, "heat_solve: allocation of thermal-discrete rates failed");
    CKR(cudaMemsetAsync(ctx->d_Dtd.p, 0, sizeof(double) * (size_t)doff[G], st));
    const double* gl = ctx->d_gl.as<double>();
    CKR(launch_cooling_window(ctx->N, ctx->d_lam.as<double>(), ctx->d_cabs.as<double>(), ctx->d_bin_off.as<int>(), G,
                              ctx->d_T.as<double>(), ctx->d_E.as<double>(), ctx->d_Dtd_woff.as<long long>(), woff[G],
                              ctx->d_Dtd_off.as<long long>(), ctx->d_Dtd.as<double>(), gl, gl + kGLPoints, st));
    CKR(cudaStreamSynchronize(st));
    ctx->td_built = true;
    return HEAT_OK;
}

// Smallest default chunk worth pipelining host copies against.
constexpr int kHostIoMinChunk = 1024;

// Default cells per chunk: as many as 45 % of the device memory the library could use (free
// memory plus the chunk scratch it already holds) allows for `nslots` chunks in flight (B band,
// X history, field tables per 32-cell group), at least one group; with several slots the range
// is also split evenly over them.  More cells per chunk means more warps in flight for the
// latency-bound build and recursion kernels.
// Whether a solve of `count` cells with these options runs the fused build + recursion.
static bool uses_fused(const heat_ctx* ctx, const heat_opts& o, int count) {
    const bool want = o.fused_build == 1 || (o.fused_build == 0 && ctx->tuned_fused);
    return o.build == HEAT_BUILD_F32 && o.heating == HEAT_HEATING_INTEGRAL && count > kSmallCells && want;
}

static int default_chunk(heat_ctx* ctx, int build, int count, int nslots, bool fused) {
    const size_t band_bytes = fused ? 0 : (size_t)ctx->band_per_cell * 32 * (build == 0 ? 8 : 4);
    const size_t per_group = band_bytes + (size_t)ctx->nbt * 32 * 10 + (size_t)ctx->N * 32 * 16;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = size_t(16) << 30;
    size_t held = 0;
    for (auto& sl : ctx->slots) held += sl.ua64.cap + sl.su64.cap + sl.ua32.cap + sl.Bb64.cap + sl.Bb32.cap + sl.xs.cap +
                                        sl.ep.cap;
    const size_t budget = std::max<size_t>(size_t(2) << 30, (size_t)(0.45 * (double)(free_b + held)));
    size_t groups = std::max<size_t>(1, budget / (size_t)nslots / per_group);
    size_t want = ((size_t)count + 31) / 32;
    if (nslots > 1) want = (want + nslots - 1) / nslots;
    return (int)(std::min(groups, std::max<size_t>(1, want)) * 32);
}

// Tail-pruning threshold as a power of two: the smallest L with 2^-L <= eps (0 = off).  The
// recursion compares binary exponents, e(a) < e(b) - L, which implies a < 2^-L b <= eps b.
static int prune_log2(double eps) {
    if (!(eps > 0.0)) return 0;
    int L = (int)std::ceil(-std::log2(eps));
    return std::max(1, std::min(L, 1000));
}

heat_status heat_solve(heat_ctx* ctx, const heat_opts* opts, double* P_out, void* j_out, void* stream) {
    if (!ctx || !opts) return HEAT_EINVAL;
    if (ctx->G == 0) return ctx->fail(HEAT_ESTATE, "heat_solve: grains not set");
    if (!ctx->u_dev && ctx->n_cells > 0) return ctx->fail(HEAT_ESTATE, "heat_solve: fields not set");
    const heat_opts& o = *opts;
    if ((o.build != HEAT_BUILD_F64 && o.build != HEAT_BUILD_F32) || o.emis < HEAT_EMIS_NONE || o.emis > HEAT_EMIS_TF32 ||
        (o.j_dtype != HEAT_F64 && o.j_dtype != HEAT_F32))
        return ctx->fail(HEAT_EINVAL, "heat_solve: bad precision option");
    if (o.heating != HEAT_HEATING_INTEGRAL && o.heating != HEAT_HEATING_POINT)
        return ctx->fail(HEAT_EINVAL, "heat_solve: bad heating option");
    if (o.heating == HEAT_HEATING_POINT && o.build != HEAT_BUILD_F64)
        return ctx->fail(HEAT_EINVAL, "heat_solve: the point rule needs the FP64 build");
    if (!(o.prune_eps >= 0.0 && o.prune_eps < 1.0))
        return ctx->fail(HEAT_EINVAL, "heat_solve: prune_eps must be in [0, 1)");
    if (o.size_integrate && !ctx->has_w) return ctx->fail(HEAT_EINVAL, "heat_solve: size integration needs weights");
    if (o.chunk_cells < 0 || (o.chunk_cells % 32) != 0)
        return ctx->fail(HEAT_EINVAL, "heat_solve: chunk_cells must be a non-negative multiple of 32");
    if (o.host_io < 0 || o.host_io > 2) return ctx->fail(HEAT_EINVAL, "heat_solve: host_io must be 0, 1 or 2");
    if (o.fused_build < 0 || o.fused_build > 2)
        return ctx->fail(HEAT_EINVAL, "heat_solve: fused_build must be 0, 1 or 2");
    if (o.recur_blocks_per_sm < 0 || o.recur_blocks_per_sm > 4)
        return ctx->fail(HEAT_EINVAL, "heat_solve: recur_blocks_per_sm must be in 0..4");
    if (o.emis_n_tile != 0 && o.emis_n_tile != 128 && o.emis_n_tile != 256)
        return ctx->fail(HEAT_EINVAL, "heat_solve: emis_n_tile must be 0, 128 or 256");
    if (o.build_prefetch < 0 || o.build_prefetch > 2)
        return ctx->fail(HEAT_EINVAL, "heat_solve: build_prefetch must be 0, 1 or 2");
    if (o.cooling != HEAT_COOLING_CONTINUOUS && o.cooling != HEAT_COOLING_DISCRETE)
        return ctx->fail(HEAT_EINVAL, "heat_solve: bad cooling option");
    const bool discrete = o.cooling == HEAT_COOLING_DISCRETE;
    if (discrete && (o.build != HEAT_BUILD_F64 || o.heating != HEAT_HEATING_INTEGRAL))
        return ctx->fail(HEAT_EINVAL, "heat_solve: thermal-discrete cooling needs the exact build and integral heating");
    if (discrete && (ctx->max_bins > kDiscreteMaxBins || td_fill_smem_bytes(ctx->N) > kMaxSmemPerBlock))
        return ctx->fail(HEAT_EINVAL, "heat_solve: thermal-discrete cooling takes at most 2048 bins per grain and "
                                      "6456 wavelengths");
    const int emis_nt = o.emis_n_tile ? o.emis_n_tile : (ctx->tuned_emis_nt ? ctx->tuned_emis_nt : 256);
    int c_begin = o.cell_begin, count = o.cell_count > 0 ? o.cell_count : ctx->n_cells - o.cell_begin;
    if (c_begin < 0 || count < 0 || c_begin + count > ctx->n_cells)
        return ctx->fail(HEAT_EINVAL, "heat_solve: cell range outside the fields");
    bool want_j = (j_out != nullptr) && o.emis != HEAT_EMIS_NONE;
    if (j_out && o.emis == HEAT_EMIS_NONE) return ctx->fail(HEAT_EINVAL, "heat_solve: j_out given with HEAT_EMIS_NONE");
    if (count == 0) return HEAT_OK;
    CKR(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int N = ctx->N, G = ctx->G, nbt = ctx->nbt;
    const int build = o.build;
    const size_t jel = o.j_dtype == HEAT_F64 ? 8 : 4;
    const size_t jrow = (size_t)(o.size_integrate ? 1 : G) * N;

    // chunks in flight and cells per chunk: the caller's, else heat_autotune's, else the
    // default: one stream, chunks as large as the memory budget allows (default_chunk),
    // since a chunk's build and recursion run faster with more warps in flight and its
    // recursion time is bounded below by its longest tasks
    int nslots = o.streams > 0 ? o.streams : 0;
    int chunk = o.chunk_cells;
    if (nslots == 0 && chunk == 0 && ctx->tuned_streams > 0) {
        nslots = ctx->tuned_streams;
        chunk = ctx->tuned_chunk;
    }
    // with synchronous host buffers the default is two chunks in flight on two streams, so
    // that one chunk's copy to the host overlaps the other's kernels (measured: ~4 % end to
    // end on the batched workload; chaining the chunks' kernels instead was slower); with
    // asynchronous host I/O the copies overlap the next call's kernels, so one chunk
    if (nslots == 0) nslots = (o.host_io == 1 && count >= 2 * kHostIoMinChunk) ? 2 : 1;
    nslots = std::min(nslots, (int)heat_ctx::kMaxSlots);
    if (chunk == 0) chunk = default_chunk(ctx, build, count, nslots, uses_fused(ctx, o, count));
    const int n_chunks = (count + chunk - 1) / chunk;
    nslots = std::max(1, std::min(nslots, n_chunks));
    const int span = std::min(count, chunk);
    const int Cc = (span + 31) / 32 * 32, NG = Cc / 32;
    const int tail_cells = count - (n_chunks - 1) * chunk;
    const int tail_NG = (tail_cells + 31) / 32;
    const bool tc = want_j && o.emis > HEAT_EMIS_F64;
    const bool si = o.size_integrate != 0;
    // the mixed path's build runs inside the recursion (no B band in memory)
    const bool fused = uses_fused(ctx, o, count);
    const int fused_nw = fused ? fused_warps(G * NG) : 0;
    if (fused && fused_nw <= 0) return ctx->fail(HEAT_ECUDA, "heat_solve: occupancy query of the fused kernel failed");

    // task lists (uploaded before any chunk is launched: nothing in the chunk loop waits for the host)
    if (ctx->tasks_NG != NG) {
        auto tasks = make_tasks(ctx, NG);
        if (ctx->s_tasks.ensure(sizeof(int2) * tasks.size()))
            return ctx->fail(HEAT_ENOMEM, "heat_solve: scratch allocation failed");
        CKR(cudaDeviceSynchronize());
        CKR(cudaMemcpy(ctx->s_tasks.p, tasks.data(), sizeof(int2) * tasks.size(), cudaMemcpyHostToDevice));
        ctx->tasks_NG = NG;
    }
    if (tail_NG != NG && ctx->tail_NG != tail_NG) {
        auto tasks = make_tasks(ctx, tail_NG);
        if (ctx->s_tasks_tail.ensure(sizeof(int2) * tasks.size()))
            return ctx->fail(HEAT_ENOMEM, "heat_solve: scratch allocation failed");
        CKR(cudaDeviceSynchronize());
        CKR(cudaMemcpy(ctx->s_tasks_tail.p, tasks.data(), sizeof(int2) * tasks.size(), cudaMemcpyHostToDevice));
        ctx->tail_NG = tail_NG;
    }
    if (tc) {
        if (!tensor_map_encoder()) return ctx->fail(HEAT_ECUDA, "heat_solve: cuTensorMapEncodeTiled unavailable");
        heat_status hs = ensure_tc_mode(ctx, o.emis, si, st);
        if (hs != HEAT_OK) return hs;
        if ((hs = prepare_tc_rows(ctx, o.emis, si, Cc)) != HEAT_OK) return hs;
    }

    // thermal-discrete: spectra solved per launch, their rate matrices within about 4 GB (two
    // resident spectra per SM at 1024 bins)
    long long td_batch = 0;
    if (discrete) {
        heat_status hs = ensure_discrete(ctx, st);
        if (hs != HEAT_OK) return hs;
        const long long per = (long long)ctx->max_bins * ctx->max_bins * (long long)sizeof(double);
        td_batch = std::max(1LL, std::min((long long)span * G, (4LL << 30) / per));
    }
    // the recursion's epilogue packs the tensor-core operand (per-grain output, lane-per-cell
    // kernels); P then goes to memory only where the caller asked for it
    const bool pack_in_recur = tc && !si && !fused && count > kSmallCells && !discrete;
    // scratch of every slot in use
    bool internal_P = (P_out == nullptr) || o.host_io;
    const bool async_io = o.host_io == 2;
    const int io_set = async_io ? ctx->io_parity : 0;
    for (int k = 0; k < nslots; ++k) {
        auto& sl = ctx->slots[k];
        bool ok = true;
        if (build == 0) {
            ok &= !sl.ua64.ensure(sizeof(double) * (size_t)N * Cc);
            ok &= !sl.su64.ensure(sizeof(double) * (size_t)N * Cc);
            if (!discrete)  // the thermal-discrete solve builds its own rate matrices
                ok &= !sl.Bb64.ensure(sizeof(double) * (size_t)NG * std::max(1LL, ctx->band_per_cell) * 32);
        } else {
            ok &= !sl.ua32.ensure(sizeof(float2) * (size_t)N * Cc);  // (u, slope) pairs
            if (fused)
                ok &= !sl.phs.ensure(sizeof(float) * (size_t)fused_nw * (N + 1) * 32);
            else
                ok &= !sl.Bb32.ensure(sizeof(float) * (size_t)NG * std::max(1LL, ctx->band_per_cell) * 32);
        }
        ok &= !sl.xs.ensure(sizeof(double) * (size_t)NG * nbt * 32);
        if (discrete) ok &= !sl.tdq.ensure(sizeof(double) * (size_t)td_batch * ctx->max_bins * ctx->max_bins);
        ok &= !sl.ep.ensure(sizeof(unsigned short) * (size_t)NG * nbt * 32);
        ok &= !sl.pabs.ensure(sizeof(double) * (size_t)Cc * G);
        ok &= !sl.work.ensure(sizeof(int) * 2);
        // staging set of this call: asynchronous host I/O alternates between two, so that one
        // call's copies to the host read a set that the next call does not write
        DevBuf& stP = io_set ? sl.P_alt : sl.P;
        DevBuf& stj = io_set ? sl.j_alt : sl.j;
        DevBuf& stl = io_set ? sl.led_alt : sl.led;
        if (internal_P) ok &= !(P_out && async_io ? stP : sl.P).ensure(sizeof(double) * (size_t)Cc * nbt);
        if (want_j && o.host_io) ok &= !stj.ensure(jel * (size_t)Cc * jrow);
        if (o.ledger_out && o.host_io) ok &= !stl.ensure(sizeof(double) * 2 * (size_t)Cc * G);
        if (tc) {
            auto& t = si ? ctx->tc_si[o.emis] : ctx->tc[o.emis];
            const int Gt = si ? 1 : G;
            ok &= !sl.A.ensure((mode_tf32(o.emis) ? 4 : 2) * (size_t)t.aoff_h[Gt]);
            ok &= !sl.rowscale.ensure(sizeof(float) * (size_t)Cc * Gt);
        }
        if (!ok) return ctx->fail(HEAT_ENOMEM, "heat_solve: scratch allocation failed");
        if (nslots > 1 && !sl.stream) {
            CKR(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
            CKR(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
        }
        if (async_io && !sl.copy) {
            CKR(cudaStreamCreateWithFlags(&sl.copy, cudaStreamNonBlocking));
            CKR(cudaEventCreateWithFlags(&sl.computed, cudaEventDisableTiming));
            for (cudaEvent_t& e : sl.copied) CKR(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        }
    }
    if (nslots > 1 && !ctx->ev_fork) CKR(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));

    GrainDev gd{};
    gd.N = N;
    gd.G = G;
    gd.nbt = nbt;
    {   // the FP32 build's pattern prefetch: the caller's setting, else the tuned one, else on for
        // grids of at most 1024 wavelengths
        const int mode = o.build_prefetch ? o.build_prefetch
                                          : (ctx->tuned_prefetch ? ctx->tuned_prefetch : (N <= 1024 ? 1 : 2));
        gd.pat_prefetch = mode == 1 ? 32 : 0;
    }
    gd.lam = ctx->d_lam.as<double>();
    gd.dln = ctx->d_dln.as<double>();
    gd.bin_off = ctx->d_bin_off.as<int>();
    gd.Cact = ctx->d_Cact.as<double>();
    gd.sC = ctx->d_sC.as<double>();
    gd.lam32 = ctx->d_lam32.as<float>();
    gd.dln32 = ctx->d_dln32.as<float>();
    gd.ca32 = ctx->d_ca32.as<float>();
    gd.ce32 = ctx->d_ce32.as<float>();
    gd.sC32 = ctx->d_sC32.as<float>();
    gd.invdE32 = ctx->d_invdE32.as<float>();
    gd.invC = ctx->d_invC.as<double>();
    gd.invdE = ctx->d_invdE.as<double>();
    gd.cde = ctx->d_cde.as<double>();
    gd.E = ctx->d_E.as<double>();
    gd.rowptr = ctx->d_rowptr.as<int>();
    gd.wmax = ctx->d_wmax.as<int>();
    gd.band_total = ctx->band_per_cell;
    gd.max_bins = ctx->max_bins;
    gd.band_max = ctx->band_max;
    gd.wmax_all = ctx->wmax_all;
    gd.seg_ptr = ctx->d_seg_ptr.as<int>();
    gd.pat64 = ctx->d_pat64.as<PatF64>();
    gd.pat32 = ctx->d_pat32.as<PatF32>();
    gd.soft = ctx->d_soft.as<SoftF64>();
    gd.soft_off = ctx->d_soft_off.as<int>();
    gd.pent = ctx->d_pent.as<PointEnt>();
    gd.pcol = ctx->d_pcol.as<int>();
    gd.kexp = ctx->d_kexp.as<int>();
    gd.rent = ctx->d_rent.as<RowEnt32>();

    // fork: every slot stream starts after the work already queued on the caller's stream
    if (nslots > 1) {
        CKR(cudaEventRecord(ctx->ev_fork, st));
        for (int k = 0; k < nslots; ++k) CKR(cudaStreamWaitEvent(ctx->slots[k].stream, ctx->ev_fork, 0));
    }
    for (int ci = 0; ci < n_chunks; ++ci) {
        const int c0 = ci * chunk;
        auto& sl = ctx->slots[ci % nslots];
        cudaStream_t cs = nslots > 1 ? sl.stream : st;
        const int cells = std::min(chunk, count - c0);
        const int cc_pad = (cells + 31) / 32 * 32;
        ChunkDev ch{};
        ch.small = count <= kSmallCells ? 1 : 0;
        ch.point = o.heating == HEAT_HEATING_POINT ? 1 : 0;
        ch.prune = prune_log2(o.prune_eps);
        ch.cells = cells;
        ch.Cc = cc_pad;
        ch.NG = cc_pad / 32;
        ch.tasks = (ch.NG == NG ? ctx->s_tasks : ctx->s_tasks_tail).as<int2>();
        ch.btasks = ch.tasks + (size_t)G * ch.NG;
        ch.n_tasks = G * ch.NG;
        ch.ua64 = sl.ua64.as<double>();
        ch.su64 = sl.su64.as<double>();
        ch.ua32 = sl.ua32.as<float>();
        ch.Bb64 = sl.Bb64.as<double>();
        ch.Bb32 = sl.Bb32.as<float>();
        ch.xs = sl.xs.as<double>();
        ch.ep = sl.ep.as<unsigned short>();
        ch.pabs = sl.pabs.as<double>();
        ch.status = ctx->d_status.as<int>();
        ch.ldP = nbt;
        DevBuf& stP = (P_out && async_io && io_set) ? sl.P_alt : sl.P;
        DevBuf& stj = io_set ? sl.j_alt : sl.j;
        DevBuf& stl = io_set ? sl.led_alt : sl.led;
        ch.P = internal_P ? stP.as<double>() : P_out + (size_t)c0 * nbt;
        if (pack_in_recur) {
            auto& t = ctx->tc[o.emis];
            ch.packA = sl.A.p;
            ch.pack_aoff = t.aoff.as<long long>();
            ch.pack_kp = t.kp.as<int>();
            ch.pack_rowscale = sl.rowscale.as<float>();
            ch.pack_tf32 = mode_tf32(o.emis) ? 1 : 0;
            ch.pack_split = mode_split(o.emis) ? 1 : 0;
            if (P_out == nullptr) ch.P = nullptr;  // nobody reads it
        }
        ch.ledger = !o.ledger_out ? nullptr
                    : (o.host_io ? stl.as<double>() : o.ledger_out + (size_t)c0 * G * 2);
        long long cell0 = (long long)c_begin + c0;
        // staging still being copied to the host by an earlier asynchronous call is not
        // written before that copy is done
        for (int k = 0; k < 2; ++k)
            if (sl.copied_valid[k] && (!async_io || k == io_set)) CKR(cudaStreamWaitEvent(cs, sl.copied[k], 0));
        ch.work = sl.work.as<int>();
        ch.blocks_per_sm = o.recur_blocks_per_sm > 0 ? o.recur_blocks_per_sm : ctx->tuned_recur_bps;
        CKR(cudaMemsetAsync(ch.work, 0, sizeof(int) * 2, cs));
        TIMED(HEAT_T_FIELD, launch_field(gd, ctx->u_dev, ctx->u_dtype, cell0, ch, build, cs));
        if (discrete) {  // field tables, then per batch the rate matrices (timed as the build) and their solve
            const long long qst = (long long)ctx->max_bins * ctx->max_bins;
            for (long long s0 = 0, nsp = (long long)ch.cells * G; s0 < nsp; s0 += td_batch) {
                const long long n = discrete_batch_spectra(gd, ch, s0, td_batch);
                TIMED(HEAT_T_BUILD, launch_discrete_fill(gd, ch, ctx->d_Dtd.as<double>(), ctx->d_Dtd_off.as<long long>(),
                                                         ctx->d_Dtd_order.as<int>(), sl.tdq.as<double>(), qst, s0, n,
                                                         cs));
                TIMED(HEAT_T_RECUR, launch_discrete_gth(gd, ch, ctx->d_Dtd_order.as<int>(), sl.tdq.as<double>(), qst, s0,
                                                        n, cs));
            }
        } else if (fused) {
            ch.phs = sl.phs.as<float>();
            TIMED(HEAT_T_RECUR, launch_fused(gd, ch, cs));
        } else {
            TIMED(HEAT_T_BUILD, launch_build(gd, ch, build, cs));
            TIMED(HEAT_T_RECUR, launch_recur(gd, ch, build, cs));
        }
        if (want_j) {
            char* jdst = o.host_io ? stj.as<char>() : (char*)j_out + (size_t)c0 * jrow * jel;
            cudaEvent_t ta = nullptr;
            if (o.timing) {
                ta = ctx->take_event();
                CKR(cudaEventRecord(ta, cs));
            }
            if (tc) {
                heat_status hs = emis_tc_chunk(ctx, o.emis, si, ch.P, cells, sl.A.p, sl.rowscale.as<float>(), jdst,
                                               o.j_dtype == HEAT_F64, pack_in_recur, emis_nt, cs);
                if (hs != HEAT_OK) return hs;
            } else if (si)
                CKR(launch_gemm_f64(cells, N, 1, ctx->d_koff_all.as<int>(), ch.P, nbt, ctx->d_Kw.as<double>(), N, jdst,
                                    N, 0, o.j_dtype == HEAT_F32, cs));
            else
                CKR(launch_gemm_f64(cells, N, G, ctx->d_bin_off.as<int>(), ch.P, nbt, ctx->d_K.as<double>(), N, jdst,
                                    (long long)G * N, N, o.j_dtype == HEAT_F32, cs));
            if (o.timing) {
                cudaEvent_t tb = ctx->take_event();
                CKR(cudaEventRecord(tb, cs));
                ctx->timed.push_back({HEAT_T_EMIS, ta, tb});
            }
        }
        // copies to the host: on the chunk's stream (host_io = 1), or on the slot's copy
        // stream after the chunk's kernels (host_io = 2)
        cudaStream_t xs = cs;
        if (async_io) {
            CKR(cudaEventRecord(sl.computed, cs));
            CKR(cudaStreamWaitEvent(sl.copy, sl.computed, 0));
            xs = sl.copy;
        }
        if (want_j && o.host_io)
            CKR(cudaMemcpyAsync((char*)j_out + (size_t)c0 * jrow * jel, stj.p, (size_t)cells * jrow * jel,
                                cudaMemcpyDeviceToHost, xs));
        if (o.ledger_out && o.host_io)
            CKR(cudaMemcpyAsync(o.ledger_out + (size_t)c0 * G * 2, ch.ledger, sizeof(double) * 2 * (size_t)cells * G,
                                cudaMemcpyDeviceToHost, xs));
        if (P_out && o.host_io)
            CKR(cudaMemcpyAsync(P_out + (size_t)c0 * nbt, ch.P, sizeof(double) * (size_t)cells * nbt,
                                cudaMemcpyDeviceToHost, xs));
        if (async_io) {
            CKR(cudaEventRecord(sl.copied[io_set], sl.copy));
            sl.copied_valid[io_set] = true;
        }
    }
    // join: the caller's stream continues after every chunk
    if (nslots > 1)
        for (int k = 0; k < nslots; ++k) {
            CKR(cudaEventRecord(ctx->slots[k].done, ctx->slots[k].stream));
            CKR(cudaStreamWaitEvent(st, ctx->slots[k].done, 0));
        }
    if (o.host_io == 1) CKR(cudaStreamSynchronize(st));
    if (async_io) ctx->io_parity ^= 1;
    return HEAT_OK;
}

heat_status heat_autotune(heat_ctx* ctx, const heat_opts* opts, double* P_out, void* j_out, void* stream,
                          int* streams_out, int* chunk_out) {
    if (!ctx || !opts) return HEAT_EINVAL;
    if (opts->host_io) return ctx->fail(HEAT_EINVAL, "heat_autotune: device buffers only");
    CKR(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int count = opts->cell_count > 0 ? opts->cell_count : ctx->n_cells - opts->cell_begin;
    struct Cand {
        int streams, chunk;
    };
    // the default (one stream, chunks as large as the scratch budget allows) first, then
    // 1-3 streams with the range cut into 1, 2, 4 or 8 chunks per stream
    std::vector<Cand> cands{{1, 0}};
    for (int sN : {1, 2, 3})
        for (int div : {1, 2, 4, 8}) {
            int chunk = ((count + sN * div - 1) / (sN * div) + 31) / 32 * 32;
            if (chunk < 256 && div > 1) continue;
            if (sN > 1 && (count + chunk - 1) / chunk < sN) continue;
            if (sN == 1 && div == 1) continue;  // the default covers it
            cands.push_back({sN, chunk});
        }
    // the launch-shape choices of an earlier tuning do not apply while these are timed
    ctx->tuned_recur_bps = ctx->tuned_emis_nt = ctx->tuned_fused = ctx->tuned_prefetch = 0;
    ctx->tuned_streams = ctx->tuned_chunk = 0;
    // each timed solve starts with a cold L2 (a write larger than L2 before it), as a solve
    // on fresh fields would
    int l2 = 0;
    CKR(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device));
    DevBuf flush;
    if (flush.ensure(std::max<size_t>(2 * (size_t)l2, 1 << 20)))
        return ctx->fail(HEAT_ENOMEM, "heat_autotune: allocation");
    cudaEvent_t e0, e1;
    CKR(cudaEventCreate(&e0));
    CKR(cudaEventCreate(&e1));
    auto done = [&](heat_status h) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return h;
    };
    // median of three cold-L2 solves of one configuration
    auto time_config = [&](const Cand& c, float* ms) -> heat_status {
        heat_opts o = *opts;
        o.streams = c.streams;
        o.chunk_cells = c.chunk;
        o.timing = 0;
        heat_status h = heat_solve(ctx, &o, P_out, j_out, stream);  // warm-up: allocations, uploads
        if (h != HEAT_OK) return h;
        float ms3[3];
        for (int rep = 0; rep < 3; ++rep) {
            if (cudaMemsetAsync(flush.p, rep, flush.cap, st) != cudaSuccess) return HEAT_ECUDA;
            if (cudaEventRecord(e0, st) != cudaSuccess) return HEAT_ECUDA;
            if ((h = heat_solve(ctx, &o, P_out, j_out, stream)) != HEAT_OK) return h;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms3[rep], e0, e1) != cudaSuccess)
                return ctx->fail(HEAT_ECUDA, "heat_autotune: timing");
        }
        std::sort(ms3, ms3 + 3);
        *ms = ms3[1];
        return HEAT_OK;
    };
    float best = 1e30f;
    Cand pick{1, 0};
    for (const Cand& c : cands) {
        float ms = 0.0f;
        heat_status h = time_config(c, &ms);
        if (h != HEAT_OK) return done(h);
        if (ms < best) {
            best = ms;
            pick = c;
        }
    }
    // then, on the chosen configuration, the recursion's task order: the weight of a row
    // against a band element in the longest-first order
    const int w0 = ctx->row_weight;
    int best_w = w0;
    for (int w : {0, 12, 30, 60}) {
        if (w == w0) continue;
        ctx->row_weight = w;
        order_grains(ctx);
        float ms = 0.0f;
        heat_status h = time_config(pick, &ms);
        if (h != HEAT_OK) return done(h);
        if (ms < best) {
            best = ms;
            best_w = w;
        }
    }
    ctx->row_weight = best_w;
    order_grains(ctx);
    // then the launch shapes, each on the configuration chosen so far (kept where faster):
    // the persistent recursion's resident blocks per SM, the tensor-core tile width and, on
    // the mixed path, the fused build + recursion kernel
    heat_status hk = HEAT_OK;
    for (int v : {3, 2}) {  // resident recursion blocks per SM (0: as many as fit)
        const int keep = ctx->tuned_recur_bps;
        ctx->tuned_recur_bps = v;
        float ms = 0.0f;
        if ((hk = time_config(pick, &ms)) != HEAT_OK) return done(hk);
        if (ms < best) best = ms; else ctx->tuned_recur_bps = keep;
    }
    if (opts->emis > HEAT_EMIS_F64 && opts->emis_n_tile == 0) {
        ctx->tuned_emis_nt = 128;
        float ms = 0.0f;
        if ((hk = time_config(pick, &ms)) != HEAT_OK) return done(hk);
        if (ms < best) best = ms; else ctx->tuned_emis_nt = 0;
    }
    if (opts->build == HEAT_BUILD_F32 && opts->heating == HEAT_HEATING_INTEGRAL && opts->fused_build == 0) {
        ctx->tuned_fused = 1;
        float ms = 0.0f;
        if ((hk = time_config(pick, &ms)) != HEAT_OK) return done(hk);
        if (ms < best) best = ms; else ctx->tuned_fused = 0;
    }
    if (opts->build == HEAT_BUILD_F32 && opts->build_prefetch == 0 && !ctx->tuned_fused) {
        ctx->tuned_prefetch = ctx->N <= 1024 ? 2 : 1;  // the other setting than the default
        float ms = 0.0f;
        if ((hk = time_config(pick, &ms)) != HEAT_OK) return done(hk);
        if (ms < best) best = ms; else ctx->tuned_prefetch = 0;
    }
    done(HEAT_OK);
    ctx->tuned_streams = pick.streams;
    ctx->tuned_chunk = pick.chunk;
    if (streams_out) *streams_out = pick.streams;
    if (chunk_out) *chunk_out = pick.chunk;
    return HEAT_OK;
}

struct heat_graph {
    heat_ctx* ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
};

heat_status heat_graph_create(heat_ctx* ctx, const heat_opts* opts, double* P_out, void* j_out, void* stream,
                              heat_graph** out) {
    if (!out) return HEAT_EINVAL;
    *out = nullptr;
    if (!ctx || !opts) return HEAT_EINVAL;
    if (opts->timing || opts->host_io) return ctx->fail(HEAT_EINVAL, "heat_graph_create: timing and host_io not allowed");
    CKR(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (st == nullptr) return ctx->fail(HEAT_EINVAL, "heat_graph_create: capture needs a non-default stream");
    // fix the chunking now: the default depends on free memory, which the warm-up changes
    heat_opts o = *opts;
    if (o.streams == 0 && o.chunk_cells == 0 && ctx->tuned_streams > 0) {
        o.streams = ctx->tuned_streams;
        o.chunk_cells = ctx->tuned_chunk;
    }
    if (o.streams == 0) o.streams = 1;
    if (o.chunk_cells == 0) {
        const int count = o.cell_count > 0 ? o.cell_count : ctx->n_cells - o.cell_begin;
        o.chunk_cells = default_chunk(ctx, o.build, std::max(count, 1), std::min(o.streams, (int)heat_ctx::kMaxSlots),
                                      uses_fused(ctx, o, count));
    }
    heat_status h = heat_solve(ctx, &o, P_out, j_out, stream);  // allocations, uploads, streams
    if (h != HEAT_OK) return h;
    CKR(cudaStreamSynchronize(st));
    CKR(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    h = heat_solve(ctx, &o, P_out, j_out, stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (h != HEAT_OK) {
        if (g) cudaGraphDestroy(g);
        return h;
    }
    if (e != cudaSuccess) return ctx->cuda_fail(e, "heat_graph_create: capture");
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return ctx->cuda_fail(e, "heat_graph_create: instantiate");
    }
    size_t n = 0;
    CKR(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    long long kernels = 0;
    if (n) {
        CKR(cudaGraphGetNodes(g, nodes.data(), &n));
        for (auto nd : nodes) {
            cudaGraphNodeType t;
            CKR(cudaGraphNodeGetType(nd, &t));
            kernels += t == cudaGraphNodeTypeKernel;
        }
    }
    heat_graph* gr = new (std::nothrow) heat_graph();
    if (!gr) {
        cudaGraphExecDestroy(x);
        cudaGraphDestroy(g);
        return HEAT_ENOMEM;
    }
    gr->ctx = ctx;
    gr->graph = g;
    gr->exec = x;
    gr->kernels = kernels;
    *out = gr;
    return HEAT_OK;
}

heat_status heat_graph_launch(heat_graph* gr, void* stream) {
    if (!gr || !gr->exec) return HEAT_EINVAL;
    heat_ctx* ctx = gr->ctx;
    CKR(cudaSetDevice(ctx->device));
    cudaError_t e = cudaGraphLaunch(gr->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? HEAT_OK : ctx->cuda_fail(e, "heat_graph_launch");
}

heat_status heat_graph_nodes(const heat_graph* gr, long long* kernel_nodes) {
    if (!gr || !kernel_nodes) return HEAT_EINVAL;
    *kernel_nodes = gr->kernels;
    return HEAT_OK;
}

void heat_graph_destroy(heat_graph* gr) {
    if (!gr) return;
    cudaSetDevice(gr->ctx->device);
    if (gr->exec) cudaGraphExecDestroy(gr->exec);
    if (gr->graph) cudaGraphDestroy(gr->graph);
    delete gr;
}

heat_status heat_sync(heat_ctx* ctx) {
    if (!ctx) return HEAT_EINVAL;
    CKR(cudaSetDevice(ctx->device));
    CKR(cudaDeviceSynchronize());
    int st = 0;
    CKR(cudaMemcpy(&st, ctx->d_status.p, sizeof(int), cudaMemcpyDeviceToHost));
    CKR(cudaMemset(ctx->d_status.p, 0, sizeof(int)));
    if (st & kStatBadInput) return ctx->fail(HEAT_EINVAL, "device: negative or non-finite field value");
    if (st & kStatNumeric) return ctx->fail(HEAT_ENUMERIC, "device: zero cooling rate with non-zero inflow");
    if (st & kStatTimeout) return ctx->fail(HEAT_ETIMEOUT, "device: bounded wait gave up");
    return HEAT_OK;
}

const char* heat_last_error(const heat_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

heat_status heat_get_tuning(const heat_ctx* ctx, heat_tuning* out) {
    if (!ctx || !out) return HEAT_EINVAL;
    out->streams = ctx->tuned_streams;
    out->chunk_cells = ctx->tuned_chunk;
    out->row_weight = ctx->row_weight;
    out->recur_blocks_per_sm = ctx->tuned_recur_bps;
    out->emis_n_tile = ctx->tuned_emis_nt;
    out->fused_build = ctx->tuned_fused;
    out->build_prefetch = ctx->tuned_prefetch;
    return HEAT_OK;
}

heat_status heat_set_wait_limit(heat_ctx* ctx, long long polls) {
    if (!ctx) return HEAT_EINVAL;
    if (polls < 0) return ctx->fail(HEAT_EINVAL, "heat_set_wait_limit: polls must be >= 0");
    ctx->wait_polls = polls;
    return HEAT_OK;
}

heat_status heat_get_cooling(heat_ctx* ctx, double* Cf) {
    if (!ctx || !Cf) return HEAT_EINVAL;
    if (ctx->G == 0) return ctx->fail(HEAT_ESTATE, "heat_get_cooling: grains not set");
    CKR(cudaSetDevice(ctx->device));
    CKR(cudaMemcpy(Cf, ctx->d_Cf.p, sizeof(double) * ctx->nbt, cudaMemcpyDeviceToHost));
    return HEAT_OK;
}

heat_status heat_get_cooling_discrete(heat_ctx* ctx, double* D) {
    if (!ctx || !D) return HEAT_EINVAL;
    if (ctx->G == 0) return ctx->fail(HEAT_ESTATE, "heat_get_cooling_discrete: grains not set");
    CKR(cudaSetDevice(ctx->device));
    heat_status h = ensure_discrete(ctx, 0);
    if (h != HEAT_OK) return h;
    size_t n = 0;
    for (int g = 0; g < ctx->G; ++g) {
        const size_t nb = (size_t)(ctx->bin_off[g + 1] - ctx->bin_off[g]);
        n += nb * nb;
    }
    std::vector<double> Dt(n);  // the device keeps each block by source bin (row u, column l)
    CKR(cudaMemcpy(Dt.data(), ctx->d_Dtd.p, sizeof(double) * n, cudaMemcpyDeviceToHost));
    size_t o = 0;
    for (int g = 0; g < ctx->G; ++g) {
        const size_t nb = (size_t)(ctx->bin_off[g + 1] - ctx->bin_off[g]);
        for (size_t l = 0; l < nb; ++l)
            for (size_t u = 0; u < nb; ++u) D[o + l * nb + u] = Dt[o + u * nb + l];
        o += nb * nb;
    }
    return HEAT_OK;
}

heat_status heat_get_timing(heat_ctx* ctx, double* ms, long long* launches, int reset) {
    if (!ctx) return HEAT_EINVAL;
    CKR(cudaSetDevice(ctx->device));
    double acc[HEAT_T_COUNT] = {0, 0, 0, 0};
    long long cnt[HEAT_T_COUNT] = {0, 0, 0, 0};
    for (auto& t : ctx->timed) {
        CKR(cudaEventSynchronize(t.b));
        float v = 0.0f;
        CKR(cudaEventElapsedTime(&v, t.a, t.b));
        acc[t.kind] += v;
        cnt[t.kind] += 1;
    }
    for (int k = 0; k < HEAT_T_COUNT; ++k) {
        if (ms) ms[k] = acc[k];
        if (launches) launches[k] = cnt[k];
    }
    if (reset) {
        for (auto& t : ctx->timed) {
            ctx->event_pool.push_back(t.a);
            ctx->event_pool.push_back(t.b);
        }
        ctx->timed.clear();
    }
    return HEAT_OK;
}

heat_status heat_band_elements(const heat_ctx* ctx, long long* per_cell) {
    if (!ctx || !per_cell) return HEAT_EINVAL;
    if (ctx->G == 0) return HEAT_ESTATE;
    *per_cell = ctx->band_per_cell;
    return HEAT_OK;
}

void heat_destroy(heat_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    DevBuf* bufs[] = {&ctx->d_lam, &ctx->d_dln, &ctx->d_lam32, &ctx->d_dln32, &ctx->d_bin_off, &ctx->d_cabs,
                      &ctx->d_T, &ctx->d_E, &ctx->d_Cf, &ctx->d_invC, &ctx->d_invdE, &ctx->d_invdE32, &ctx->d_Cact,
                      &ctx->d_sC, &ctx->d_ca32, &ctx->d_ce32, &ctx->d_sC32, &ctx->d_rowptr, &ctx->d_wmax, &ctx->d_seg_ptr,
                      &ctx->d_pat64, &ctx->d_pat32, &ctx->d_soft, &ctx->d_soft_off, &ctx->d_K, &ctx->d_Kw, &ctx->d_w,
                      &ctx->d_koff_all, &ctx->d_cde, &ctx->d_pent, &ctx->d_pcol, &ctx->d_kexp, &ctx->d_rent, &ctx->d_gl, &ctx->d_Dtd, &ctx->d_Dtd_off, &ctx->d_Dtd_woff, &ctx->d_Dtd_order, &ctx->d_u_own, &ctx->s_tasks, &ctx->s_tasks_tail, &ctx->d_status};
    for (DevBuf* b : bufs) b->release();
    for (auto& sl : ctx->slots) {
        DevBuf* sb[] = {&sl.ua64, &sl.su64, &sl.ua32, &sl.Bb64, &sl.Bb32, &sl.xs, &sl.ep,   &sl.pabs,
                        &sl.P,    &sl.j,    &sl.led,  &sl.A,    &sl.rowscale, &sl.work, &sl.P_alt, &sl.j_alt,
                        &sl.led_alt, &sl.phs, &sl.tdq};
        for (DevBuf* b : sb) b->release();
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.copy) cudaStreamDestroy(sl.copy);
        if (sl.computed) cudaEventDestroy(sl.computed);
        for (cudaEvent_t e : sl.copied)
            if (e) cudaEventDestroy(e);
    }
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    for (auto* modes : {ctx->tc, ctx->tc_si})
        for (int m = 0; m < 5; ++m) {
            modes[m].B.release();
            modes[m].colscale.release();
            modes[m].kp.release();
            modes[m].boff.release();
            modes[m].aoff.release();
        }
    surrogate_free(ctx->sur);
    ctx->sur = nullptr;
    for (auto& t : ctx->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    delete ctx;
}

}  // extern "C"

// Internal (not part of the C ABI): read-only view of a ctx's grain tables for the
// no-allocation solve in noalloc.cu.
__attribute__((visibility("hidden"))) heat_status heat_internal_grain_view(heat_ctx* ctx, GrainDev* gd, int* device,
                                                                           int** status) {
    if (!ctx) return HEAT_EINVAL;
    if (ctx->G == 0) return ctx->fail(HEAT_ESTATE, "heat_solve_noalloc: grains not set");
    *gd = GrainDev{};  // every field set below or left zero (no pattern prefetch)
    gd->N = ctx->N;
    gd->G = ctx->G;
    gd->nbt = ctx->nbt;
    gd->lam = ctx->d_lam.as<double>();
    gd->dln = ctx->d_dln.as<double>();
    gd->bin_off = ctx->d_bin_off.as<int>();
    gd->Cact = ctx->d_Cact.as<double>();
    gd->sC = ctx->d_sC.as<double>();
    gd->lam32 = ctx->d_lam32.as<float>();
    gd->dln32 = ctx->d_dln32.as<float>();
    gd->ca32 = ctx->d_ca32.as<float>();
    gd->ce32 = ctx->d_ce32.as<float>();
    gd->sC32 = ctx->d_sC32.as<float>();
    gd->invdE32 = ctx->d_invdE32.as<float>();
    gd->invC = ctx->d_invC.as<double>();
    gd->invdE = ctx->d_invdE.as<double>();
    gd->cde = ctx->d_cde.as<double>();
    gd->E = ctx->d_E.as<double>();
    gd->rowptr = ctx->d_rowptr.as<int>();
    gd->wmax = ctx->d_wmax.as<int>();
    gd->band_total = ctx->band_per_cell;
    gd->max_bins = ctx->max_bins;
    gd->band_max = ctx->band_max;
    gd->wmax_all = ctx->wmax_all;
    gd->seg_ptr = ctx->d_seg_ptr.as<int>();
    gd->pat64 = ctx->d_pat64.as<PatF64>();
    gd->pat32 = ctx->d_pat32.as<PatF32>();
    gd->soft = ctx->d_soft.as<SoftF64>();
    gd->soft_off = ctx->d_soft_off.as<int>();
    gd->pent = ctx->d_pent.as<PointEnt>();
    gd->pcol = ctx->d_pcol.as<int>();
    gd->kexp = ctx->d_kexp.as<int>();
    gd->rent = ctx->d_rent.as<RowEnt32>();
    *device = ctx->device;
    *status = ctx->d_status.as<int>();
    return HEAT_OK;
}

__attribute__((visibility("hidden"))) void heat_internal_fail(heat_ctx* ctx, const char* msg) {
    if (ctx) ctx->err = msg;
}
