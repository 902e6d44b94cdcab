/*
 * heat.h -- C ABI of libheat: stochastic heating and emissivity of dust grains
 * on one NVIDIA GB300 (sm_103a).
 *
 * The method is Porter & Vladimirov, "Calculation of Stochastic Heating and
 * Emissivity of Cosmic Dust Grains ..." (HEATCODE), Sec. 2:
 *   - enthalpy bins i = 0..M with centres E_i = H(T_i)            (Sec. 2.1)
 *   - heating elements T_ul, u > l, from Omega = u_lambda C_abs with
 *     log-log interpolation between wavelength nodes                (Eq. heating, Eq. interpolation)
 *   - thermal-continuous cooling T_{f-1,f}                           (Eq. adjacent, Eq. cooling)
 *   - B_fj = sum_{k>=f} T_kj and the X recursion, then P = X / sum X (Eq. bmatrix, Eq. xf, Eq. renormalization)
 *   - emissivity j_lambda = C_abs(lambda) sum_i P_i B_lambda(T_i) [E_i >= hc/lambda]
 *                                                                    (Eq. emission, Eq. emission-lambda)
 *   - optional size integration J = sum_g w_g j_g                    (Eq. convolution)
 * The heating element is the wavelength integral over the target bin's edges,
 *   T_ul = (1/h) int Omega(lambda) lambda dlambda over [hc/(Ehi_u - E_l), hc/(Elo_u - E_l)],
 * with Elo_0 = 0, Elo_i = (E_{i-1}+E_i)/2, Ehi_i = Elo_{i+1}, Ehi_M = infinity, plus the
 * power of photons too soft to leave bin l carried by T_{l+1,l}.  Cooling integrates the
 * cross-section continued as a power law beyond the wavelength grid.
 *
 * Units are CGS: wavelengths in cm, u_lambda in erg cm^-3 cm^-1, C_abs in cm^2,
 * temperatures in K, enthalpies in erg, P dimensionless, j in erg s^-1 sr^-1 cm^-1.
 *
 * Conventions for every call:
 *   - A heat_ctx is bound to one CUDA device; calls on one ctx must not run
 *     concurrently from several host threads (distinct ctxs are independent).
 *   - Host arrays are read during the call only.  Device pointers are borrowed:
 *     they must stay valid until the work queued on the given stream completes.
 *   - Argument errors return HEAT_EINVAL synchronously and queue no work.
 *   - Errors detected on the device (non-finite input, a zero cooling rate with
 *     non-zero inflow) are recorded in a device status word and reported by
 *     heat_sync (and by the next call that synchronises).
 *   - heat_last_error returns a message for the last failed call on the ctx.
 */
#ifndef LIBHEAT_HEAT_H
#define LIBHEAT_HEAT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct heat_ctx heat_ctx;

typedef enum {
    HEAT_OK = 0,
    HEAT_EINVAL = 1,   /* bad argument; nothing queued */
    HEAT_ENOMEM = 2,   /* device or host allocation failed */
    HEAT_ECUDA = 3,    /* a CUDA call failed (message in heat_last_error) */
    HEAT_ENUMERIC = 4, /* a cooling rate is zero while the bin receives inflow (no steady state) */
    HEAT_ETIMEOUT = 5, /* a bounded device-side wait gave up */
    HEAT_ESTATE = 6    /* call out of order (e.g. solve before grains/fields are set) */
} heat_status;

/* element types for field input and emissivity output */
enum { HEAT_F64 = 0, HEAT_F32 = 1 };

/* precision of the matrix build (B elements and the per-cell wavelength tables);
 * the recursion (Eq. xf) always accumulates in FP64 */
enum { HEAT_BUILD_F64 = 0, HEAT_BUILD_F32 = 1 };

/* heating matrix (Eq. heating) */
enum {
    HEAT_HEATING_INTEGRAL = 0, /* each element integrates the photon rate over the upper bin's edges
                                  (plus the intra-bin term of sub-bin photons); B telescopes to
                                  one cumulative integral per element                             */
    HEAT_HEATING_POINT = 1     /* the paper's point rule: T_ul = Omega(lambda_ul) lambda_ul^3 dE_u
                                  / (h^2 c) at lambda_ul = hc / (E_u - E_l), Omega on the log-log
                                  interpolant (Eq. interpolation), dE_u the upper bin's width (the
                                  top bin takes E_M - E_{M-1}), no intra-bin term; B by suffix sums
                                  down each column (Eq. brecurrence).  Exact build only          */
};

/* cooling transitions (Sec. 2.1: the thermal approximations beside Eq. adjacent) */
enum {
    HEAT_COOLING_CONTINUOUS = 0, /* thermal-continuous: only the adjacent downward transition, rate
                                    Eq. cooling; P by the Guhathakurta-Draine recursion (Eq. xf)   */
    HEAT_COOLING_DISCRETE = 1    /* thermal-discrete: a grain in bin u emits as a body at T_u and a
                                    photon of energy e takes it to the bin l holding E_u - e; the
                                    rate to l is the power of Eq. cooling's integrand in that photon-
                                    energy window divided by E_u - E_l (photons too soft to leave
                                    bin u go with the adjacent transition), so that the rates carry
                                    Eq. cooling's power.  P by the stationary solve of the full rate
                                    matrix (Eq. steady-state, Eq. level-sum; state reduction,
                                    up to M^3/3 multiply-adds per spectrum, fewer where the rates
                                    span few bins).  Needs the exact build (HEAT_BUILD_F64), the
                                    integral heating form, at most 2048 bins per grain and 6456
                                    wavelengths (HEAT_EINVAL otherwise); the downward rates are
                                    computed on the first such solve after heat_set_grains       */
};

/* emissivity contraction (Eq. emission) */
enum {
    HEAT_EMIS_NONE = -1,  /* no emissivity */
    HEAT_EMIS_F64 = 0,    /* FP64 FMA contraction (exact path) */
    HEAT_EMIS_BF16X3 = 1, /* tensor cores: P and K scaled by powers of two per (cell, grain) row and
                             per (grain, wavelength) column, split into BF16 hi + lo, three products
                             (hi*hi + hi*lo + lo*hi) accumulated in FP32 */
    HEAT_EMIS_TF32X3 = 2, /* same with TF32 hi + lo */
    HEAT_EMIS_BF16 = 3,   /* single BF16 product (hi*hi), FP32 accumulation */
    HEAT_EMIS_TF32 = 4    /* single TF32 product, FP32 accumulation */
};

typedef struct heat_opts {
    int build;          /* HEAT_BUILD_F64 (exact) or HEAT_BUILD_F32 (mixed)                      */
    int emis;           /* HEAT_EMIS_*                                                             */
    int j_dtype;        /* HEAT_F64 or HEAT_F32 element type of j_out                              */
    int size_integrate; /* 0: j_out is [cells][grains][n_lambda]; 1: [cells][n_lambda], sum_g w_g j_g
                           (tensor-core modes: one GEMM over all grains' bins, the sum is formed
                           in the accumulator)                                                    */
    int cell_begin;     /* first cell solved (0-based)                                             */
    int cell_count;     /* cells solved; <= 0 means all cells from cell_begin                      */
    int chunk_cells;    /* cells per internal chunk (multiple of 32; 0 = library default: as many
                           as 45 % of the usable device memory holds)                             */
    int host_io;        /* 1: P_out, j_out and ledger_out are host pointers; the library stages
                           through device memory and the call returns after the results are on
                           the host.  2: the same, asynchronous: the call returns once the work is
                           queued, the copies to the host run on an internal copy stream and the
                           host buffers are complete after heat_sync (which waits for the device);
                           the device staging alternates between two sets, so the copies of one
                           call overlap the kernels of the next (a pipelined loop: set the next
                           fields, solve, ...; heat_sync before reading the results of the last
                           two calls).  cuda_stream continues after the kernels, not the copies */
    int timing;         /* 1: record CUDA events around every kernel launch (see heat_get_timing)  */
    double* ledger_out; /* NULL, or FP64 [cell_count][n_grains][2] (device; host with host_io): the
                           energy check of every spectrum, erg/s: [0] absorbed power c int u C dlambda
                           on the grid, [1] emitted power of the discrete model
                           sum_f P_f T_{f-1,f} (E_f - E_{f-1}) (Eq. cooling); they differ by the
                           bin discretisation of the absorbed photon energies only                */
    int streams;        /* chunks in flight (1..4), each on an internal stream forked from and
                           joined back into cuda_stream, so that the recursion of one chunk
                           overlaps the matrix build and emissivity of the next; 0 = the
                           library default (heat_autotune's choice, else 1 on device buffers, 2
                           with host_io = 1, whose copies then overlap the other chunk's kernels,
                           and 1 with host_io = 2).
                           Results do not depend on it or on chunk_cells, except that solves of
                           at most 16 cells take element-parallel kernels (same bounds against
                           the oracle, rounding differs in the last bits)                      */
    int heating;        /* HEAT_HEATING_INTEGRAL (default) or HEAT_HEATING_POINT (needs
                           HEAT_BUILD_F64).  The ledger's absorbed power [0] is the physical one
                           either way, so with the point rule [1]/[0] shows what the rule loses */
    double prune_eps;   /* 0 (default): every bin is solved.  eps in (0, 1): tail pruning, an
                           approximation in the spirit of the paper's level cut-off (appendix,
                           algorithm optimisations: pruning):
                           a spectrum's recursion stops once every bin of the current row's band
                           window has X_i below 2^-L of the largest X so far and X_i Kmax_i below
                           2^-L of the largest such product (Kmax_i = max over the grid of
                           C_abs B_lambda(T_i); 2^-L <= eps, compared on binary exponents), and
                           P of the bins above is 0.  Those bins carry less than about eps of the
                           probability and of j_lambda at any wavelength relative to its peak.
                           Results still do not depend on chunking or grouping.  Outside [0, 1):
                           HEAT_EINVAL                                                          */
    int fused_build;    /* 1: on the mixed path (HEAT_BUILD_F32, integral heating, more than 16
                           cells) the matrix build runs inside the recursion kernel and the B band
                           never exists in memory (4 bytes per band element and cell less scratch,
                           so larger default chunks); timed as HEAT_T_RECUR with no HEAT_T_BUILD
                           launches.  2: a build kernel writes the B band to device memory, then
                           the recursion reads it.  0 (default): heat_autotune's choice if it made
                           one, else 2.  Elsewhere it is ignored.  Results are bit-identical either
                           way.  On a GB300 the fused kernel is slower (it issues the build's
                           instructions in the recursion's warps)                               */
    int recur_blocks_per_sm; /* resident blocks per SM of the persistent recursion (1..4); 0 = as many
                           as fit (heat_autotune's choice if it made one).  Fewer leave room on
                           every SM for another chunk's build kernel when chunks are in flight on
                           several streams.  Results do not depend on it                        */
    int emis_n_tile;    /* wavelength columns of a tensor-core emissivity tile: 256 or 128 (tiles are
                           128 cells x this; the operand ring holds 4 or 6 k-stages); 0 =
                           heat_autotune's choice, else 256.  Results do not depend on it        */
    int cooling;        /* HEAT_COOLING_CONTINUOUS (default) or HEAT_COOLING_DISCRETE          */
    int build_prefetch; /* FP32 matrix build (more than 16 cells, not fused): 1: each segment step
                           prefetches into L1 the pattern entry 32 entries past the segment's end;
                           2: no prefetch; 0 (default): heat_autotune's choice if it made one, else
                           1 on grids of at most 1024 wavelengths and 2 above (measured on a GB300:
                           4.19 -> 3.89 ms per step of the 4096-cell x 64-grain x 1024-wavelength
                           workload, 71.4 -> 86.9 ms of the 65536-cell x 32-grain x 2048-wavelength
                           one).  Results do not depend on it                                 */
} heat_opts;

/* kernel classes reported by heat_get_timing */
enum {
    HEAT_T_FIELD = 0, /* field transpose and u slopes                     */
    HEAT_T_BUILD = 1, /* matrix build: B band (Eq. bmatrix) and intra-bin terms; with
                         thermal-discrete cooling, the full rate matrices                */
    HEAT_T_RECUR = 2, /* band-limited recursion and renormalisation (Eq. xf); with
                         thermal-discrete cooling, the state reduction and normalisation */
    HEAT_T_EMIS = 3,  /* emissivity contraction (Eq. emission)              */
    HEAT_T_COUNT = 4
};

/* Fill *opts with defaults: exact FP64 build, FP64 emissivity, FP64 j, per-grain j,
 * all cells, device outputs, no timing, no energy check. */
void heat_default_opts(heat_opts* opts);

/* Create a context on CUDA device `device` for the wavelength grid lambda_cm[n_lambda]
 * (host, strictly ascending, > 0, n_lambda >= 2).  The grid is copied.
 * Errors: HEAT_EINVAL (bad grid), HEAT_ECUDA, HEAT_ENOMEM. */
heat_status heat_create_grid(heat_ctx** out, int device, int n_lambda, const double* lambda_cm);

/* Set the grain sizes (Sec. 2; paper's GrainModel + temperature grid).  All arrays are host:
 *   radius_cm[n_grains]              grain radius (kept for size bookkeeping; > 0)
 *   c_abs_cm2[n_grains][n_lambda]    absorption cross-section on the grid (>= 0, finite)
 *   bin_offset[n_grains+1]           bins of grain g are bin_offset[g] .. bin_offset[g+1]-1,
 *                                    at least 2 and at most 4096 bins per grain
 *   T_bins_K[bin_offset[n_grains]]   bin temperatures, strictly ascending per grain, > 0
 *   H_bins_erg[bin_offset[n_grains]] bin enthalpies E_i = H(T_i), strictly ascending per grain, > 0
 *   size_weight[n_grains] or NULL    weights w_g for size integration (Eq. convolution)
 * Computes on the device, once: cooling rates (Eq. cooling, FP64 Gauss-Legendre),
 * the Planck kernels C_abs B_lambda(T_i) [E_i >= hc/lambda], and the field-independent
 * band tables of each grain (which (f, j) can be reached by a photon on the grid, and
 * where each transition wavelength hc/(Elo_f - E_j) falls on the grid).
 * Synchronous.  Errors: HEAT_EINVAL, HEAT_ENOMEM, HEAT_ECUDA. */
heat_status heat_set_grains(heat_ctx* ctx, int n_grains, const double* radius_cm, const double* c_abs_cm2,
                            const int* bin_offset, const double* T_bins_K, const double* H_bins_erg,
                            const double* size_weight);

/* Enthalpy bins on a temperature grid (Sec. 2: the bins sit on a user-supplied temperature
 * grid, E_i = H(T_i); Sec. 2.1: the enthalpy is the integral of the grain's heat capacity):
 * the Debye internal energy of 3 n_atoms modes above the zero-point energy,
 *   H(T) = 9 n_atoms k T (T / theta_D)^3 int_0^{theta_D/T} x^3 / (e^x - 1) dx   (erg),
 * the integral summed in closed series (Bernoulli series below theta_D/T = 1, exponential
 * series above), relative accuracy about 1e-14.  theta_D in K (> 0), n_atoms > 0, T in K
 * (>= 0; H(0) = 0); all finite, else NaN.  Host function: no ctx, no device, thread-safe.
 * Limits: (3 pi^4 / 5) n_atoms k T^4 / theta_D^3 for T << theta_D; 3 n_atoms k T -
 * (9/8) n_atoms k theta_D for T >> theta_D. */
double heat_debye_enthalpy(double theta_D, double n_atoms, double T);

/* Measured FMA throughput of `device` (a diagnostic for rooflines; no ctx): fp64 = 1 for FP64
 * fused multiply-adds, 0 for FP32.  Runs independent FMA chains on every SM at full
 * occupancy (a few ms of device time on the legacy stream, after the device's earlier work)
 * and writes the rate in TFLOP/s (2 flop per FMA) to *tflops (host pointer).
 * Errors: HEAT_EINVAL (null pointer, negative device), HEAT_ECUDA. */
heat_status heat_measure_fma_peak(int device, int fp64, double* tflops);

/* Set the radiation fields u_lambda[n_cells][n_lambda] (erg cm^-3 cm^-1, >= 0, finite),
 * element type `dtype` (HEAT_F64 or HEAT_F32).  on_device = 1: `u_lambda` is a device
 * pointer, borrowed until the solves that use it complete; on_device = 0: host memory
 * (pinned or pageable), copied asynchronously on `stream` into library-owned device memory.
 * Negative or non-finite values are flagged on the device during heat_solve
 * (HEAT_EINVAL from heat_sync).  Errors: HEAT_EINVAL, HEAT_ENOMEM, HEAT_ECUDA, HEAT_ESTATE. */
heat_status heat_set_fields(heat_ctx* ctx, int n_cells, const void* u_lambda, int dtype, int on_device,
                            void* cuda_stream);

/* Solve cells [cell_begin, cell_begin + cell_count) on `cuda_stream` (a cudaStream_t, NULL = legacy):
 *   P_out  FP64 [cell_count][bin_offset[n_grains]] or NULL: the steady-state distributions
 *          P of every grain (Eq. renormalization), row c holds all grains' bins back to back;
 *   j_out  j_dtype, [cell_count][n_grains][n_lambda] (or [cell_count][n_lambda] with
 *          size_integrate) or NULL: the emissivity (Eq. emission).
 * Device pointers unless opts->host_io.  Asynchronous with respect to the host unless
 * host_io = 1; device-side errors surface at heat_sync.  Non-interacting grains give
 * P = delta_{i0} (no error).  P entries below the normal FP64 range (about 2.2e-308) are
 * returned as 0.  Errors: HEAT_EINVAL, HEAT_ESTATE, HEAT_ENOMEM, HEAT_ECUDA. */
heat_status heat_solve(heat_ctx* ctx, const heat_opts* opts, double* P_out, void* j_out, void* cuda_stream);

/* Time heat_solve on cells [opts->cell_begin, +opts->cell_count) of the current fields for
 * a set of (streams, chunk_cells) pairs (the default first; each timed solve after a write
 * larger than L2; the median of three) and keep the fastest: later solves whose opts leave
 * both at 0 use it.  *streams_out / *chunk_out (or NULL) receive the choice (chunk 0 = the
 * default size).  Then, on that configuration, it times the recursion's task order (grains
 * longest first by band elements + w x rows, w in {0, 12, 30, 60}; 30 before tuning) and
 * keeps the fastest w for all later solves on the ctx (heat_set_grains resets it).  Then, one
 * at a time on the configuration chosen so far, the launch shapes: the persistent recursion's
 * resident blocks per SM (all, 3, 2), for tensor-core emissivity the tile width (256 or 128
 * wavelengths), for the mixed path the fused build + recursion kernel and the FP32 build's
 * pattern prefetch (the other setting than the default); each kept if faster.
 * heat_get_tuning reports the choice; solves whose opts leave a knob at 0 use it.  Results
 * do not depend on any of them.  Runs the candidates on cuda_stream and synchronises; j_out / P_out as in
 * heat_solve (device, with room for the cells), overwritten.  Allocates a temporary buffer
 * of twice the L2 size.  Errors: as heat_solve. */
heat_status heat_autotune(heat_ctx* ctx, const heat_opts* opts, double* P_out, void* j_out, void* cuda_stream,
                          int* streams_out, int* chunk_out);

/* ---- CUDA graphs ----------------------------------------------------------------------
 * A solve captured once and replayed: the launch cost of a solve's kernels (field, build,
 * recursion, packing, emissivity per chunk) is paid once, which matters for small solves
 * (a single cell's grains) and for solves repeated over changing fields (an iterative
 * radiative-transfer loop that updates u in place).
 * heat_graph_create runs heat_solve(ctx, opts, P_out, j_out) once on cuda_stream (so that
 * every allocation, upload and internal stream exists), waits for it, then captures the
 * same solve into a graph.  The graph is bound to the buffers of that call: P_out, j_out,
 * the fields pointer current at capture (heat_set_fields with on_device = 1: its contents
 * may change between launches, the pointer may not) and the ctx's scratch.  A later
 * heat_solve on the ctx with another configuration may reallocate that scratch: destroy
 * and recreate the graph after one.  opts->timing and opts->host_io are not allowed.
 * Errors: HEAT_EINVAL, HEAT_ESTATE, HEAT_ENOMEM, HEAT_ECUDA (capture refused). */
/* The configuration heat_autotune chose for the ctx (all 0 before it ran; 0 = the default). */
typedef struct heat_tuning {
    int streams, chunk_cells;  /* chunks in flight and cells per chunk                            */
    int row_weight;            /* the recursion's longest-first order: band + row_weight x rows   */
    int recur_blocks_per_sm;   /* resident blocks per SM of the persistent recursion              */
    int emis_n_tile;           /* tensor-core emissivity tile width (wavelengths)                 */
    int fused_build;           /* 1: the mixed path's build runs inside the recursion             */
    int build_prefetch;        /* the FP32 build's pattern prefetch (1 on, 2 off; 0: the default) */
} heat_tuning;
heat_status heat_get_tuning(const heat_ctx* ctx, heat_tuning* out);

typedef struct heat_graph heat_graph;
heat_status heat_graph_create(heat_ctx* ctx, const heat_opts* opts, double* P_out, void* j_out, void* cuda_stream,
                              heat_graph** out);
/* Replay the captured solve on cuda_stream (asynchronous; errors surface at heat_sync). */
heat_status heat_graph_launch(heat_graph* graph, void* cuda_stream);
/* Kernel nodes in the graph (the solve's launches). */
heat_status heat_graph_nodes(const heat_graph* graph, long long* kernel_nodes);
void heat_graph_destroy(heat_graph* graph);

/* Wait for all work of the ctx's last calls and return the device status:
 * HEAT_OK, HEAT_ENUMERIC, HEAT_EINVAL (bad field values) or HEAT_ECUDA.  Clears the status. */
heat_status heat_sync(heat_ctx* ctx);

/* Give-up limit of the device-side waits (failure detection).  The tensor-core kernels
 * (emissivity, surrogate GEMMs) hand tiles between a copy role, an MMA role and an epilogue
 * role through shared-memory barriers; a role that has polled a barrier `polls` times without
 * the other role arriving gives up: it records HEAT_ETIMEOUT in the device status word (seen
 * by heat_sync), tells the other roles to stop, waits for the copies and MMAs it already
 * issued to finish, frees its tensor memory and returns, so the context stays usable; the
 * outputs of that launch are undefined.  polls = 0 makes every such wait give up at once
 * (a test of this path); the default, HEAT_WAIT_POLLS_DEFAULT, is far above any wait of a
 * healthy launch.  Applies to launches queued after the call.  Errors: HEAT_EINVAL (polls < 0). */
#define HEAT_WAIT_POLLS_DEFAULT (1LL << 22)
heat_status heat_set_wait_limit(heat_ctx* ctx, long long polls);

/* Message of the last failure on ctx (never NULL; "" when none). */
const char* heat_last_error(const heat_ctx* ctx);

/* Copy the cooling rates T_{f-1,f} (Eq. cooling) of all grains to host Cf[bin_offset[n_grains]]
 * (Cf[bin_offset[g]] = 0 for every grain).  Errors: HEAT_ESTATE, HEAT_ECUDA. */
heat_status heat_get_cooling(heat_ctx* ctx, double* Cf_host);

/* Copy the thermal-discrete downward rates (HEAT_COOLING_DISCRETE) to host D_host: grain by
 * grain an nb_g x nb_g block, row l, column u, holding T_lu for l < u (0 elsewhere), blocks
 * back to back (sum_g nb_g^2 doubles).  Computes them first if no discrete solve has.
 * Errors: HEAT_ESTATE (grains not set), HEAT_ENOMEM, HEAT_ECUDA. */
heat_status heat_get_cooling_discrete(heat_ctx* ctx, double* D_host);

/* Number of band elements (f, j), j < f, that a photon on the grid can reach, summed over
 * grains: the FP64 FMAs of one spectrum set's recursion.  Errors: HEAT_ESTATE. */
heat_status heat_band_elements(const heat_ctx* ctx, long long* per_cell);

/* Device time per kernel class, summed over the launches recorded by solves with
 * opts->timing = 1 since the last reset: ms[HEAT_T_COUNT] (milliseconds, CUDA events on
 * the launching stream) and launches[HEAT_T_COUNT].  Waits for the recorded events.
 * reset = 1 clears the record afterwards.  Errors: HEAT_ECUDA. */
heat_status heat_get_timing(heat_ctx* ctx, double* ms, long long* launches, int reset);

/* ---- Learned surrogate (an extension: the paper's method has no surrogate) ------------
 * An ensemble of MLPs maps the binned field and the grain to ln j_lambda; it is trained on
 * spectra the exact path computes, and the exact path stays its fallback.
 * Network per member: 128 inputs (ln of the power the grain absorbs in 64 wavelength bands,
 * ln radius, a composition flag, ln of the total absorbed power, zero padding; standardised
 * with training-set statistics) -> 4 hidden layers of 512 with GELU (tanh form) -> n_lambda outputs
 * y = ln j - ln P_abs (P_abs = c int u C dlambda, standardised per wavelength).  BF16
 * operands on the tensor cores, FP32 accumulation and FP32 master weights; masked MSE
 * (entries with j < 1e-6 of the spectrum's peak are left out) plus a one-sided square penalty
 * on masked entries predicted above that level; Adam.  Requires n_lambda to be a multiple of
 * 64 and at most 4096, and FP64 device fields. */

/* Create (or recreate) the surrogate of ctx: `members` ensemble members (1..8), weights
 * initialised from `seed`; grain_flag[n_grains] (host, or NULL = 0) is the composition input.
 * Errors: HEAT_ESTATE (grains not set), HEAT_EINVAL, HEAT_ENOMEM, HEAT_ECUDA. */
heat_status heat_surrogate_init(heat_ctx* ctx, int members, const float* grain_flag, unsigned long long seed);

/* Samples of cells [cell_begin, cell_begin + cell_count), ordered (cell, grain), all device:
 *   X   FP32 [cell_count * n_grains][128] raw inputs;
 *   Y   FP32 [cell_count * n_grains][n_lambda] targets ln j - ln P_abs (NaN where masked), or NULL;
 *       needs j (FP32 [cell_count][n_grains][n_lambda], e.g. from heat_solve) when given;
 *   lnp FP32 [cell_count * n_grains] ln P_abs, or NULL.
 * Synchronous.  Errors: HEAT_ESTATE, HEAT_EINVAL, HEAT_ENOMEM, HEAT_ECUDA. */
heat_status heat_surrogate_samples(heat_ctx* ctx, int cell_begin, int cell_count, const float* j, float* X, float* Y,
                                   float* lnp, void* cuda_stream);

/* Standardisation statistics (per input, per wavelength) from n training samples. */
heat_status heat_surrogate_fit_norm(heat_ctx* ctx, const float* X, const float* Y, long long n, void* cuda_stream);

/* Train every member for `epochs` over the n samples (device X, Y) in shuffled batches of
 * `batch` rows (a multiple of 64), Adam with a learning rate decaying from lr to lr/100 on a
 * cosine over the call's steps; loss_history[epochs] (host, or NULL) receives member 0's
 * mean loss per epoch (standardised units).  Synchronous. */
heat_status heat_surrogate_train(heat_ctx* ctx, const float* X, const float* Y, long long n, int batch, int epochs,
                                 float lr, unsigned long long seed, double* loss_history, void* cuda_stream);

/* Ensemble prediction for n samples (device X and lnp from heat_surrogate_samples):
 * lnj FP32 [n][n_lambda] = ln j (ensemble mean), spread FP32 [n] = the largest ensemble
 * standard deviation of ln j over the predicted emission (within 1e-6 of its peak). */
heat_status heat_surrogate_predict(heat_ctx* ctx, const float* X, const float* lnp, long long n, float* lnj,
                                   float* spread, void* cuda_stream);

/* Surrogate with exact fallback for the cells of fallback_opts (cell_begin, cell_count):
 * j_out FP32 device [cells][n_grains][n_lambda] = exp(ln j) of the ensemble; every cell with
 * a grain whose spread exceeds tol is solved again by heat_solve with fallback_opts (its
 * exact/mixed precision choices; per-grain FP32 device j required) and overwritten.
 * fallback_opts->ledger_out (device FP64 [cells][n_grains][2], or NULL) receives the energy
 * check of every spectrum returned: for the surrogate's, [absorbed power c int u C dlambda,
 * 4 pi int j dlambda on the grid (trapezoid)]; for the cells solved exactly, heat_solve's
 * ledger.  *n_fallback = cells solved exactly.  fallback_opts->heating must be
 * HEAT_HEATING_INTEGRAL (the form the network is trained on), else HEAT_EINVAL.  Synchronous. */
heat_status heat_solve_surrogate(heat_ctx* ctx, const heat_opts* fallback_opts, float tol, float* j_out,
                                 int* n_fallback, void* cuda_stream);

/* Gradient check support: loss and gradient of member `member` for n (multiple of 64)
 * already standardised samples (device Xn [n][128], Tn [n][n_lambda], NaN = masked); the
 * gradient is written to grad_out (device FP32, flat layout: for each layer W [out][in]
 * then b [out]); *loss_out = masked mean squared error. */
heat_status heat_surrogate_grads(heat_ctx* ctx, int member, const float* Xn, const float* Tn, int n,
                                 float* grad_out, double* loss_out, void* cuda_stream);

/* Copy member parameters (flat FP32 layout above) to host (set = 0) or from host (set = 1);
 * *nparams = their count.  host may be NULL to query the count. */
heat_status heat_surrogate_params(heat_ctx* ctx, int member, float* host, int set, long long* nparams);

/* Checkpoint: weights, Adam moments, step, seed, standardisation (save); load recreates the
 * surrogate from such a file (the grid and grain count must match). */
heat_status heat_surrogate_save(heat_ctx* ctx, const char* path);
heat_status heat_surrogate_load(heat_ctx* ctx, const char* path);

/* ---- Solve without allocating (the paper has no counterpart) -------------------------
 * For callers that cannot allocate device memory once their loop runs: codes that keep
 * the GPU under a fixed memory budget owned by their own allocator, and time-critical
 * loops that cannot pay for cudaMalloc/cudaFree, which wait for the whole device to go
 * idle and so stall every other stream.  Such callers create the ctx, set the grains
 * (which allocates) once up front, then call this in the loop.
 *
 * Computes P exactly as heat_solve does (same kernels, same results) for the FP64 fields
 * u_dev[n_cells][n_lambda] (device) into P_out[n_cells][bin_offset[n_grains]] (device, FP64),
 * with build = HEAT_BUILD_F64 or HEAT_BUILD_F32, on `cuda_stream`; no emissivity.  It uses
 * no memory but the caller's buffers, the ctx's grain tables and one static device array of
 * HEAT_NOALLOC_SCRATCH_BYTES that every GPU which loads the library keeps until exit; it
 * calls no allocating routine.
 *   - The first call on each device looks up the array's device address with that device
 *     current (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - All calls on a device share the array and it keeps the last call's contents: calls
 *     whose work overlaps on the GPU (other streams or host threads) race.  Serialise them.
 *   - Cells are processed in groups of 32; one group needs
 *       band*32*(8 bytes FP64 build | 4 bytes FP32 build) + nbt*32*10 + N*32*(16 | 8) + G*8 + 2304
 *     bytes (band = heat_band_elements, G grains, N wavelengths, nbt total bins).  If that
 *     exceeds the array, the call
 *     returns HEAT_EINVAL with a message (heat_last_error) and queues nothing.
 *   - Cells run in a plain grain-major task order with one warp per task: the results equal
 *     heat_solve's, but without heat_solve's longest-first persistent scheduling the call
 *     can take longer on grain sets of very uneven bin counts.
 * Errors: HEAT_EINVAL, HEAT_ESTATE (grains not set), HEAT_ECUDA, each with a message in
 * heat_last_error; device-side errors at heat_sync.  When a call fails after it has queued
 * work for some groups of cells (a later launch failing), P_out is partly written: treat
 * its contents as undefined after any error. */
#define HEAT_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
heat_status heat_solve_noalloc(heat_ctx* ctx, int build, const double* u_dev, int n_cells, double* P_out,
                               void* cuda_stream);

/* Release the ctx and all device memory it owns (no-op on NULL). */
void heat_destroy(heat_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
