/*
 * rtt.h -- C ABI of librtt.so, the B300 (sm_103a) implementation of the
 * multi-order retarded-time imaging operator A, its adjoint A^T, and the
 * batched applies behind the operational-rank / reach / innovation audit and
 * the TSVD / ridge estimators of "Photon-Ring Retarded-Time Tomography"
 * (arXiv 2609.05528).
 *
 * General rules (apply to every entry point):
 *  - Every function returns an rtt_status; no exception crosses the ABI.
 *    On failure rtt_last_error() returns a message for the calling thread.
 *  - Pointers named *_dev are device memory of the current CUDA device,
 *    pointers named *_host are host memory.  The caller owns every buffer it
 *    passes; the library owns the operator (tables, index arrays, scratch) and
 *    frees it in rtt_destroy.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Applies are
 *    asynchronous on that stream; functions that return host results
 *    synchronise the stream before returning.
 *  - Results are deterministic: repeated calls give bitwise-identical output
 *    (no floating-point atomics; fixed summation order).
 *  - Layouts.  Source coefficients x[s][k][b]: node s = i_r * n_phi + j_phi
 *    (radius-major, azimuth contiguous), hat k (k = 0 youngest), batch b
 *    innermost.  Data y[row][f][b]: rows sorted by (order, pixel) and
 *    restricted to the orders of arm_mask, frame f, batch b innermost.
 *  - arm_mask selects image orders: bit n = order n (n = 0, 1, 2).
 *    Direct-only = 0x1, resolved stack = 0x7 (Eq. 3).
 */
#ifndef RTT_H
#define RTT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RTT_ABI_VERSION 2

typedef enum rtt_status {
    RTT_OK = 0,
    RTT_EINVAL = -1,          /* invalid argument, size or table content */
    RTT_ENOMEM = -2,          /* device or host allocation failed */
    RTT_ECUDA = -3,           /* a CUDA runtime call failed */
    RTT_ETIMEOUT = -4,        /* a bounded device wait gave up */
    RTT_ENOTCONVERGED = -5,   /* an iteration hit its limit */
    RTT_ESTATE = -6,          /* call not valid in the operator's state */
    RTT_EDEVICE = -7          /* a device-side consistency check failed */
} rtt_status;

typedef struct rtt_op_s* rtt_op;

/* Kerr spin a (|a| < 1, M = 1) and observer inclination in degrees
   (0 < incl < 90).  The observer azimuth is 0. */
typedef struct {
    double spin;
    double incl_deg;
} rtt_geometry;

/* Equatorial source grid: n_r radii log-spaced on [r_in, r_out] (n_r >= 2),
   n_phi azimuths phi_j = 2 pi j / n_phi (n_phi >= 2, periodic). */
typedef struct {
    int32_t n_r;
    int32_t n_phi;
    double r_in;
    double r_out;
} rtt_source_grid;

/* Observer frames t_o(f) = t0 + cadence f, f < n_frames.  Hats
   B_k(t) = max(0, 1 - |t - t_k| / hat_step), t_k = t_end - hat_step k,
   k < n_hats.  cadence / hat_step must be a dyadic rational p / 2^24 with
   0 < cadence <= hat_step (exact per-frame hat offsets). */
typedef struct {
    int32_t n_frames;
    double t0;
    double cadence;
    int32_t n_hats;
    double hat_step;
    double t_end;
} rtt_time_grid;

/* Raw ray table (FP64 SoA, host memory, read during rtt_build_operator only).
   One entry per valid (screen sample, order): order in {0,1,2}; pixel >= 0
   (rows are the distinct (order, pixel) pairs); source radius r in
   [r_in, r_out] and azimuth phi (any real, taken modulo 2 pi) of the
   equatorial crossing; delay Delta (M); whitened transfer weight
   w = g^3 sqrt(dOmega_p) / S_p (Eq. 16 at sigma_Omega = 1); throughput
   g^3 dOmega_p / S_p (weights of the direct age quantile, Sec. 4.5). */
typedef struct {
    int64_t n_rays;
    const int8_t* order;
    const int32_t* pixel;
    const double* r;
    const double* phi;
    const double* delay;
    const double* weight;
    const double* throughput;
} rtt_ray_table;

/* Writable table of the same layout (output of rtt_trace_rays). */
typedef struct {
    int64_t capacity;
    int8_t* order;
    int32_t* pixel;
    double* r;
    double* phi;
    double* delay;
    double* weight;
    double* throughput;
} rtt_ray_buffer;

typedef struct {
    double snr0;  /* SNR_0 of Eq. 17-18 (> 0); scale = snr0 / s_ref */
    double rho;   /* detection threshold rho (> 0), Eq. 30-31 */
} rtt_options;

/* Summary of a built operator. */
typedef struct {
    int64_t n_rays;
    int64_t n_rows;
    int64_t rows_per_order[3];
    int64_t n_nodes;
    int32_t n_hats;
    int32_t n_frames;
    double s_ref;          /* Eq. 17 */
    double scale;          /* snr0 / s_ref: whitening factor applied by A */
    double delay_min[3];   /* per order, over its rays (NaN if no rays); of the
                              whole table for a row shard */
    double delay_max[3];
    int64_t total_rows;      /* rows of the whole table (= n_rows unless sharded) */
    int64_t total_rows_per_order[3];
    int64_t shard_row_begin; /* first row of this operator in the whole table */
    int32_t shard_index;     /* 0 and 1 unless built by rtt_build_operator_shard */
    int32_t shard_count;
    int32_t weight_precision; /* RTT_WEIGHTS_FP32 or RTT_WEIGHTS_BF16 */
    int32_t reserved;
} rtt_op_info;

/* Row shard: block `index` of `count` of the (order, pixel)-sorted rows. */
typedef struct {
    int32_t index;  /* 0 <= index < count */
    int32_t count;  /* >= 1 */
} rtt_shard;

/* Screen samples for the tracer: pixel centres or sub-rays (alpha, beta) in
   M, the pixel each belongs to and the number of sub-rays of that pixel. */
typedef struct {
    int64_t n;
    const double* alpha;
    const double* beta;
    const int32_t* pixel;
    const int32_t* n_sub;
    double d_omega_pixel;  /* pixel solid angle in M^2 */
} rtt_screen;

/*
 * rtt_error_string -- a static description of a status code;
 * rtt_last_error -- the message of the last failing call (thread-local
 * buffer owned by the library, overwritten by the next failure);
 * rtt_abi_version -- the version of this interface (1).  Library plumbing:
 * the paper has no counterpart.  Each never fails.
 */
const char* rtt_error_string(rtt_status s);
const char* rtt_last_error(void);
int rtt_abi_version(void);

/*
 * rtt_trace_rays -- null geodesics on the GPU (FP64, Mino-time Carter
 * equations in s = 1/r, u = cos theta; Sec. 3.1 Eq. 2 and Sec. 5), and the
 * raw ray table they define: for each sample and order n = 0, 1, 2 (the
 * (n+1)-th equatorial crossing, counted while the ray stays outside
 * r_+ + 0.01 M), valid if r in [r_in, r_out]; redshift of a prograde
 * Keplerian emitter outside the ISCO and an emitter plunging from the ISCO
 * inside it; delays relative to the earliest direct ray.
 * screen: host arrays.  out: host buffer with capacity >= 3 * screen->n.
 * *n_out receives the number of entries, sorted by (order, pixel, sample).
 * Errors: RTT_EINVAL (geometry, sizes, capacity), RTT_ECUDA, RTT_ENOMEM.
 */
rtt_status rtt_trace_rays(const rtt_geometry* geom, const rtt_source_grid* grid,
                          const rtt_screen* screen, rtt_ray_buffer* out, int64_t* n_out,
                          void* stream);

/*
 * rtt_arm_table -- the ray table of a Sec. 6.4 mechanism arm, built from a
 * resolved table (host code, no device work).  kind:
 *   RTT_ARM_PAIRING_DESTROYED: within each order n, with the order's rays
 *     listed by ascending index (i_0 < i_1 < ...) and again by ascending
 *     (keys_host, index) (j_0, j_1, ...), ray i_m takes the delay of ray j_m:
 *     each order keeps its delays, their pairing with source point and
 *     weight is broken.  keys_host: n_rays finite doubles (the random draw,
 *     supplied by the caller).
 *   RTT_ARM_DELAY_ONLY: each ring ray (order >= 1) takes the source point
 *     (r, phi) of its direct quantile partner and keeps its delay.
 *   RTT_ARM_SPATIAL_ONLY: each ring ray takes the delay of its direct
 *     quantile partner and keeps its source point.
 * The direct quantile partner of the ray of rank k (by delay, ties by index)
 * among the E_n rays of order n is the direct ray of rank
 * floor((k + 1/2) E_0 / E_n) among the E_0 direct rays.  in: the resolved
 * table (host; only order, r, phi and delay are read).  r_out, phi_out,
 * delay_out: host arrays of n_rays doubles owned by the caller (they may
 * alias the input columns); the other columns of the arm's table are the
 * input's.  keys_host is ignored for the delay-only and spatial-only arms.
 * Errors: RTT_EINVAL (null pointers, unknown kind, order outside {0,1,2},
 * non-finite delay or key, no direct ray), RTT_ENOMEM.
 */
#define RTT_ARM_PAIRING_DESTROYED 1
#define RTT_ARM_DELAY_ONLY 2
#define RTT_ARM_SPATIAL_ONLY 3
rtt_status rtt_arm_table(int kind, const rtt_ray_table* in, const double* keys_host,
                         double* r_out, double* phi_out, double* delay_out);

/*
 * rtt_build_operator -- packs a raw FP64 ray table into the device operator
 * (Sec. 3.1 Eq. 2-3; Eq. 16 weights; Eq. 17-18 normalisation): bilinear
 * corner weights in (log r, phi) premultiplied by w (FP32, derived in FP64),
 * integer hat base and 24-bit hat fraction per ray (derived in FP64, so that
 * the set of hats touched equals the exact one), the row CSR over rays
 * sorted by (order, pixel) on the device, and the adjoint's tables of rays
 * by source cell.  Computes s_ref with j_ref = 1 evaluated directly and
 * scale = snr0 / s_ref.
 * table: host FP64 SoA (not retained).  *out receives the handle.
 * Errors: RTT_EINVAL (bad grid, non-dyadic cadence/hat_step, order outside
 * {0,1,2}, negative pixel, r outside [r_in, r_out], non-finite values, no
 * direct ray), RTT_ENOMEM, RTT_ECUDA.
 */
rtt_status rtt_build_operator(const rtt_geometry* geom, const rtt_source_grid* grid,
                              const rtt_time_grid* time, const rtt_ray_table* table,
                              const rtt_options* opt, void* stream, rtt_op* out);

/*
 * rtt_build_operator_shard -- the operator restricted to one block of rows
 * (Sec. 3.1: each row of the stack of Eq. 3 is the response of one (order,
 * pixel) to the whole source, so a block of rows is an operator of its own).
 * shard == NULL or count == 1: the whole operator (rtt_build_operator).
 * Otherwise every rank passes the WHOLE raw table; shard `index` of `count`
 * keeps rows [R index / count, R (index + 1) / count) of the R sorted rows
 * (rtt_shard_rows) and their rays, with s_ref and scale of the whole table,
 * so the shards' A x are the whole operator's rows, bit for bit, and the
 * whole A^T y is the sum over shards of each shard's A^T of its rows.
 * On a shard, the applies, rtt_probe_info, rtt_gram, rtt_gram_class and
 * rtt_gram_normal sum over the shard's rows only (the whole operator's value
 * is the sum over shards); entry points that need every row (order mixing,
 * the direct age quantile, reach, the rank audit, the solvers) return
 * RTT_ESTATE.  arm_mask still selects orders: a shard's y holds its own rows
 * of the selected orders, in order.
 * Errors: those of rtt_build_operator; RTT_EINVAL for an invalid shard or a
 * shard with no rows (count > R).
 */
rtt_status rtt_build_operator_shard(const rtt_geometry* geom, const rtt_source_grid* grid,
                                    const rtt_time_grid* time, const rtt_ray_table* table,
                                    const rtt_options* opt, const rtt_shard* shard, void* stream,
                                    rtt_op* out);

/*
 * rtt_set_weight_precision -- precision of the corner weights the FP32
 * applies use (Eq. 2 bilinear weights times the whitened ray weight of
 * Eq. 16 and the scale of Eq. 18; no counterpart in the paper, which works in
 * FP64).  RTT_WEIGHTS_FP32 (the default): each weight is its FP64 value
 * rounded to FP32.  RTT_WEIGHTS_BF16: that FP32 value rounded on to BF16
 * (nearest even); the fast kernels then read an 8-byte BF16 copy per ray
 * instead of 16 bytes, and every kernel variant computes the same operator
 * bit for bit.  The FP64 applies always use the FP64 weights.  Synchronises
 * `stream`.
 * Errors: RTT_EINVAL (null op, unknown precision), RTT_ENOMEM, RTT_ECUDA.
 */
#define RTT_WEIGHTS_FP32 0
#define RTT_WEIGHTS_BF16 1
rtt_status rtt_set_weight_precision(rtt_op op, int precision, void* stream);

/*
 * rtt_shard_rows -- rows [*begin_out, *end_out) that shard `index` of `count`
 * holds out of n_rows sorted rows (the rows of the stack of Eq. 3):
 * floor(n_rows index / count) to floor(n_rows (index + 1) / count).  Host
 * only.
 * Errors: RTT_EINVAL (null pointer, n_rows < 0, invalid shard).
 */
rtt_status rtt_shard_rows(int64_t n_rows, const rtt_shard* shard, int64_t* begin_out,
                          int64_t* end_out);

/*
 * rtt_op_query -- the sizes, delay ranges and whitening of a built operator
 * (s_ref of Eq. 17, scale = SNR_0 / s_ref of Eq. 18).  out: host struct.
 * Errors: RTT_EINVAL (null op or out).
 */
rtt_status rtt_op_query(rtt_op op, rtt_op_info* out);

/*
 * rtt_arm_rows -- the number of data rows of the orders selected by arm_mask
 * (the blocks of the stack of Eq. 3; bit n selects order n), i.e. the first
 * extent of every y buffer of that arm.  rows_out: host int64.
 * Errors: RTT_EINVAL (null op or rows_out, arm_mask not in 1..7).
 */
rtt_status rtt_arm_rows(rtt_op op, int arm_mask, int64_t* rows_out);

/*
 * rtt_op_status -- the operator's device status word, read after the work
 * queued on `stream` (synchronises it).  Bit 0: a kernel's bounded wait on
 * an asynchronous copy (the TMA-staged adjoint) ran out of iterations; that
 * apply's output is incomplete.  0 after correct operation.  clear != 0
 * resets the word.  The paper has no counterpart.  flags_out: host int32.
 * Errors: RTT_EINVAL, RTT_ECUDA.
 */
rtt_status rtt_op_status(rtt_op op, int32_t* flags_out, int clear, void* stream);

/*
 * rtt_apply_A -- y = scale * A x for a batch of `batch` histories (Eq. 2-3,
 * Eq. 16, Eq. 47): y[row][f][b] = scale sum_{e in row} w_e sum_c bil_c(e)
 * sum_k B_k(t_o(f) - Delta_e) x[node_c(e)][k][b].  Only the two hats whose
 * support contains each sample are touched.
 * x_dev: float [n_nodes][n_hats][batch]; y_dev: float
 * [arm_rows][n_frames][batch] (fully overwritten).  FP32 storage and FP32
 * accumulation.  Errors: RTT_EINVAL (null pointers, batch < 1, arm_mask not
 * in 1..7), RTT_ECUDA.
 */
rtt_status rtt_apply_A(rtt_op op, const float* x_dev, float* y_dev, int batch, int arm_mask,
                       void* stream);

/*
 * rtt_apply_AT -- x = scale * A^T y, the exact transpose of rtt_apply_A
 * (Sec. 5: explicit adjoint action), evaluated as a deterministic gather
 * over the transposed node -> (ray, corner) index with no atomics.
 * y_dev: float [arm_rows][n_frames][batch]; x_dev: float
 * [n_nodes][n_hats][batch] (fully overwritten).  Errors as rtt_apply_A.
 */
rtt_status rtt_apply_AT(rtt_op op, const float* y_dev, float* x_dev, int batch, int arm_mask,
                        void* stream);

/* FP64 storage and FP64 arithmetic versions of the two applies (Eq. 2-3
   and the adjoint action of Sec. 5; the plain FP64 GPU path the fast path is
   compared with).  Same layouts in double.  Errors as rtt_apply_A. */
rtt_status rtt_apply_A_f64(rtt_op op, const double* x_dev, double* y_dev, int batch,
                           int arm_mask, void* stream);
rtt_status rtt_apply_AT_f64(rtt_op op, const double* y_dev, double* x_dev, int batch,
                            int arm_mask, void* stream);

/*
 * rtt_apply_A_AT -- the forward and adjoint pair of the reconstruction loss
 * L(x) = 1/2 ||scale A x - d||^2 (Eq. 2-3 and the explicit adjoint action of
 * Sec. 5): y = scale * A x and g = scale * A^T (y - d) = grad L, in one call.
 * x_dev: float [n_nodes][n_hats][batch]; d_dev: float [arm_rows][n_frames]
 * [batch] or NULL (then g = scale * A^T y); y_dev: float [arm_rows][n_frames]
 * [batch] (written; may be NULL only when the arm has no rows); g_dev: float
 * [n_nodes][n_hats][batch] (written).  The forward runs, y - d is formed in
 * an operator-owned scratch that grows on demand (when d is given), and the
 * adjoint runs on it: the bits of rtt_apply_A followed by rtt_apply_AT on
 * (y - d) rounded to FP32.  Asynchronous on `stream`.
 * Errors: RTT_EINVAL, RTT_ENOMEM, RTT_ECUDA.
 */
rtt_status rtt_apply_A_AT(rtt_op op, const float* x_dev, const float* d_dev, float* y_dev,
                          float* g_dev, int batch, int arm_mask, void* stream);

/*
 * rtt_probe_info -- age information of the scalar probe (Sec. 3.3 Eq. 10-12,
 * Sec. 4.4 Eq. 29): I(a) = || C^{-1/2} A_arm q_a ||^2 with
 * q_a = 1_[r_in, r_out](r) / N_h exp(-(t + a)^2 / (2 h^2)),
 * N_h^2 = pi (r_out^2 - r_in^2) h sqrt(pi), evaluated directly at each ray's
 * source point.  ages_host: n_ages (<= 256) probe ages in M; h > 0 (the
 * paper uses 3 M); info_host receives n_ages doubles.  Exponentials are
 * evaluated in FP32 and reduced in FP64; ages whose value lies within 1e-3
 * (relative) of rho^2 are re-evaluated entirely in FP64, so the pass/fail
 * decision I(a) >= rho^2 is taken at FP64 accuracy.  Synchronous.
 * Errors: RTT_EINVAL, RTT_ENOMEM, RTT_ECUDA.
 */
rtt_status rtt_probe_info(rtt_op op, int arm_mask, int n_ages, const double* ages_host, double h,
                          double* info_host, void* stream);

/*
 * rtt_probe_info_noalloc -- the FP32 pass of rtt_probe_info, with the same
 * arguments and result, for callers that must not allocate device memory
 * while they run: for example an application whose pool allocator has
 * reserved all free device memory up front, or a runtime that forbids
 * allocation after initialisation.  The paper has no counterpart: this entry
 * point only changes where the scratch lives.
 * The per-block partial sums use a file-scope static device array of
 * 1184 x 256 doubles (about 2.4 MB) that every GPU which loads the library
 * holds until the process exits; no cudaMalloc / cudaFree (or allocating
 * library routine) is called.  ages_dev (n_ages doubles) and info_dev
 * (n_ages doubles, receives I(a)) are device memory owned by the caller;
 * 0 <= n_ages <= 256, larger counts are rejected with RTT_EINVAL.  The call
 * is asynchronous on `stream` and does not perform the FP64 re-evaluation of
 * near-threshold ages that rtt_probe_info does.
 * The first call on each device looks the array's device address up with
 * cudaGetSymbolAddress (with that device current), so make that first call
 * before any stream capture begins.  All calls share the one array and each
 * call overwrites every entry it reads, so no clearing is needed; calls that
 * overlap on the GPU (for example on two streams) race on it and must be
 * serialised by the caller.
 * Errors: RTT_EINVAL (null or invalid arguments, n_ages above 256),
 * RTT_ECUDA (the symbol lookup or the launch failed).
 */
rtt_status rtt_probe_info_noalloc(rtt_op op, int arm_mask, int n_ages, const double* ages_dev,
                                  double h, double* info_dev, void* stream);

/*
 * rtt_direct_age_quantile -- the direct order's throughput-weighted age
 * boundary A_{0,q} (Sec. 4.5): over all direct (ray, frame) samples with
 * age Delta_e - t_o(f) and weight = the ray's throughput, the smallest sample
 * age whose cumulative weight (ages ascending, device radix sort, FP64
 * prefix sum) reaches q times the total.  0 < q <= 1.  Synchronous.
 * Errors: RTT_EINVAL (null op or out_host, q outside (0, 1]), RTT_ENOMEM,
 * RTT_ECUDA.
 */
rtt_status rtt_direct_age_quantile(rtt_op op, double q, double* out_host, void* stream);

typedef struct {
    int32_t anchor_index; /* youngest fully supported age, -1 if none */
    double anchor_age;    /* NaN if none */
    double L_anchor;      /* anchor-connected passing span (M) */
    double T_reach;       /* oldest passing age (Eq. 30), NaN if none */
    double A0q;           /* boundary used for J_old */
    double J_old;         /* age_step * sum_{a > A0q} log(1 + I(a)) (Eq. 35) */
} rtt_reach_result;

/*
 * rtt_reach -- historical reach and old-age innovation from I(a)
 * (Sec. 3.3 Eq. 13, Sec. 4.4 Eq. 30, Sec. 4.5 Eq. 35).  pass(a) <=>
 * I(a) >= rho^2.  The anchor is the smallest age whose support
 * [-a - 3h, -a + 3h] lies inside the union of the arm's footprints
 * W_n = [t_o,min - Delta_n^max, t_o,max - Delta_n^min]; L_anchor =
 * a_last - anchor for the contiguous passing run starting at the anchor (0
 * if the anchor fails or is absent).  J_old uses the rectangle rule with
 * strict a > a0q.  ages/info: host arrays of n_ages; pass_host (optional)
 * receives n_ages bytes.  Host-only computation.
 * Errors: RTT_EINVAL (null op, out, ages or info, n_ages < 1, h or
 * age_step not positive, arm_mask not in 1..7).
 */
rtt_status rtt_reach(rtt_op op, int arm_mask, int n_ages, const double* ages_host,
                     const double* info_host, double h, double a0q, double age_step,
                     rtt_reach_result* out, uint8_t* pass_host);

#define RTT_CLASS_S224 0 /* Eq. 8: 4 radial B-splines x 7 azimuthal x 8 DCT-II */
#define RTT_CLASS_L224 1 /* Sec. 7: the temporal DCT modes replaced by 8 hats */
/* the nested ladder of Sec. 7-8 (Eq. 43): (radial, azimuthal, temporal) */
#define RTT_CLASS_S448T 2   /* (4, 7, 16 DCT-II) */
#define RTT_CLASS_S528S 3   /* (6 cubic B-splines, 11, 8 DCT-II) */
#define RTT_CLASS_S1056ST 4 /* (6, 11, 16 DCT-II) */
#define RTT_CLASS_L448 5    /* (4, 7, 16 degree-one B-splines) */
#define RTT_CLASS_L1056 6   /* (6, 11, 16 degree-one B-splines) */
/* rtt_class_dim -- the dimension d of class `kind` (Eq. 8, Eq. 43; 0 for an
   unknown kind).  Pure function, never fails. */
int rtt_class_dim(int kind);

/*
 * rtt_synth_class -- representation class `kind` at the operator's source
 * nodes (Sec. 3.2 Eq. 5-8; Sec. 7-8 Eq. 43): Q[(s, k)][c] = R_i(r_s)
 * Phi_l(phi_s) tau_m(t_k), c = (i * NA + l) * NT + m, with NR clamped cubic
 * B-splines on uniform knots in log r (NR = 4: no interior knot), NA
 * azimuthal functions {1, cos m phi, sin m phi}, NT temporal DCT-II modes (S
 * classes) or degree-one B-splines (L classes) on the hat window [t_{K-1},
 * t_0]; columns unnormalised.  Q_dev: double [n_nodes][n_hats][d], d =
 * rtt_class_dim(kind), written asynchronously on `stream`.
 * Errors: RTT_EINVAL (unknown kind, fewer than 2 hats), RTT_ECUDA.
 */
rtt_status rtt_synth_class(rtt_op op, int kind, double* Q_dev, void* stream);

/*
 * rtt_gram -- restricted Gram matrix G = P^T P of P = scale * A_arm Q
 * (Sec. 3.2 Eq. 7, Sec. 4.1 Eq. 21): Q_dev is the class synthesis matrix in
 * the source layout, double [n_nodes][n_hats][d] (column j = direction j);
 * G_dev receives double [d][d] (symmetric, row-major).  FP64 throughout: P
 * is formed chunk by chunk by the FP64 forward kernel into library scratch
 * (<= 1 GiB) and reduced in a fixed order.  1 <= d <= 4096.  Synchronous.
 * Errors: RTT_EINVAL (null op, Q_dev or G_dev, d outside 1..4096, arm_mask
 * not in 1..7), RTT_ENOMEM, RTT_ECUDA.
 */
rtt_status rtt_gram(rtt_op op, int arm_mask, const double* Q_dev, int d, double* G_dev,
                    void* stream);

/*
 * rtt_gram_normal -- the same G = P^T P computed as G = Q^T (A^T (A Q)) through
 * the normal operator, FP64 throughout (FP64 forward and adjoint kernels on
 * 32 columns at a time, then an FP64 GEMM Q^T Z in cuBLAS).  The contraction
 * runs over n_nodes * n_hats coefficients rather than arm_rows * n_frames
 * data samples.  Same arguments and result as rtt_gram up to rounding;
 * library scratch <= 32 columns of data and coefficients.  Synchronous.
 */
/*
 * rtt_gram_class -- the same restricted Gram G = P^T P (Eq. 7, FP64, 224 x
 * 224 into G_dev) for the separable class `kind` (RTT_CLASS_S224 or
 * RTT_CLASS_L224, the columns of rtt_synth_class) without forming P or Q:
 * with s_e the class's spatial functions interpolated at ray e (times its
 * weight) and C_row the frame sums of products of the temporal functions
 * interpolated at each ray's hat coordinates, G = sum over rows and ray pairs
 * of (s_e s_e'^T) kron C_row.  About 7x fewer FP64 operations than
 * rtt_gram_normal.  Rows with more than 4 rays are not handled
 * (RTT_ESTATE; use rtt_gram_normal).  Allocates scratch; synchronous.
 * Errors: RTT_EINVAL, RTT_ESTATE, RTT_ENOMEM, RTT_ECUDA.
 */
rtt_status rtt_gram_class(rtt_op op, int arm_mask, int kind, double* G_dev, void* stream);

/*
 * rtt_gram_normal -- the restricted Gram through the normal operator,
 * G = Q^T (scale^2 A_arm^T A_arm) Q (Eq. 7, Eq. 21): Q's columns go through
 * the FP64 forward and adjoint applies in chunks and the final contraction
 * with Q^T is a cuBLAS DGEMM.  Arguments as rtt_gram.  Synchronous.
 * Errors: RTT_EINVAL (null op, Q_dev or G_dev, d outside 1..4096, arm_mask
 * not in 1..7), RTT_ENOMEM, RTT_ECUDA.
 */
rtt_status rtt_gram_normal(rtt_op op, int arm_mask, const double* Q_dev, int d, double* G_dev,
                           void* stream);

/*
 * Order mixing (Sec. 3.1 Eq. 4): d_L = C_L^{-1/2} (L (x) I) d_R with
 * C_L = (L (x) I) C_R (L^T (x) I) and C_R = I (the rows of A are whitened),
 * so a mixed arm carries the noise propagated from the resolved rows, not a
 * level of its own (Sec. 4.2).
 *   RTT_MIX_UNRESOLVED: the unresolved image -- per pixel, the sum of the
 *     arm's rows of that pixel over the orders (orders ascending) divided by
 *     the square root of their count; one output row per pixel of the arm,
 *     pixels ascending.
 *   RTT_MIX_TOTAL_FLUX: the total-flux readout -- the sum of every row of the
 *     arm (fixed row blocks summed in order, then the blocks' sums in a fixed
 *     lane split and shuffle tree) divided by the square root of the row
 *     count; one output row.
 * rtt_mix_rows_count: the mixed row count of (arm_mask, mode).
 * rtt_mix_rows(_f64): y_dev [arm rows][n_frames][batch] -> yl_dev [mixed
 *   rows][n_frames][batch] (device buffers, caller-owned, not aliased).
 * rtt_mix_rows_T(_f64): the adjoint W^T, yl_dev -> y_dev (every arm row
 *   written: the row's mixed row times the same 1 / sqrt(count)).
 * Sums run in a fixed order (bitwise repeatable).  The first call for an arm
 * mask builds that arm's pixel groups (device allocation, synchronous); the
 * total-flux scratch grows on demand (synchronous once); otherwise
 * asynchronous on `stream`.
 * Errors: RTT_EINVAL (mode, arm mask, batch < 1, null pointer), RTT_ENOMEM,
 * RTT_ECUDA.
 */
#define RTT_MIX_UNRESOLVED 1
#define RTT_MIX_TOTAL_FLUX 2
rtt_status rtt_mix_rows_count(rtt_op op, int arm_mask, int mode, int64_t* n_out);
rtt_status rtt_mix_rows(rtt_op op, int arm_mask, int mode, const float* y_dev, float* yl_dev,
                        int batch, void* stream);
rtt_status rtt_mix_rows_T(rtt_op op, int arm_mask, int mode, const float* yl_dev, float* y_dev,
                          int batch, void* stream);
rtt_status rtt_mix_rows_f64(rtt_op op, int arm_mask, int mode, const double* y_dev,
                            double* yl_dev, int batch, void* stream);
rtt_status rtt_mix_rows_T_f64(rtt_op op, int arm_mask, int mode, const double* yl_dev,
                              double* y_dev, int batch, void* stream);

/*
 * rtt_probe_info_mix -- probe information of a mixed arm (Eq. 4 with Eq.
 * 10-12, 29): I_L(a) = || W scale A q_a ||^2, W the whitened collapse of
 * `mode` over the arm's rows and q_a the scalar age probe of rtt_probe_info
 * evaluated at each ray's source point.  The arm's probe responses are formed
 * in FP64 for 16 ages at a time (terms with exponent below -100 dropped),
 * collapsed by W and squared and summed in a fixed order.  ages_host /
 * info_host: host arrays of n_ages (1..4096); h > 0.  The result feeds
 * rtt_reach for the mixed arm's reach and J_old.  Allocates device scratch
 * (arm rows x frames x 16 doubles, twice); synchronous.
 * Errors: RTT_EINVAL, RTT_ENOMEM, RTT_ECUDA.
 */
rtt_status rtt_probe_info_mix(rtt_op op, int arm_mask, int mode, int n_ages,
                              const double* ages_host, double h, double* info_host, void* stream);

/*
 * rtt_probe_info_local -- per-direction information of the 28-direction
 * localized probe class (Sec. 3.3 Eq. 14): q_{a,l} = psi_l(r, phi) / N_{h,l}
 * exp(-(t + a)^2 / (2 h^2)), psi_l = R_i(r) Phi_m(phi) (l = 7 i + m; R_i
 * the cubic Bernstein polynomials in the log-radius coordinate, Phi_m in
 * {1, cos phi, sin phi, cos 2 phi, sin 2 phi, cos 3 phi, sin 3 phi}), each
 * of unit L2 norm under r dr dphi dt; I_l(a) = || scale A_arm q_{a,l} ||^2,
 * the diagonal of the age-local Fisher matrix.  Evaluated at each ray's
 * source point, FP64, per row through the rays' Gaussian overlap sums (rows
 * of at most 4 rays; terms with exponent below -100 dropped), fixed-order
 * reductions.  info_host: host [n_ages][28].  The localized directional
 * reach is the oldest age at which some I_l(a) >= rho^2.  Allocates device
 * scratch; synchronous.  Errors: RTT_EINVAL, RTT_ESTATE (a row with more than
 * 4 rays), RTT_ENOMEM, RTT_ECUDA.
 */
rtt_status rtt_probe_info_local(rtt_op op, int arm_mask, int n_ages, const double* ages_host,
                                double h, double* info_host, void* stream);

/*
 * rtt_gram_normal_mix -- the restricted Gram of a mixed arm (Eq. 4, Eq. 7):
 * G = Q^T A^T W^T W A Q with W the whitened collapse of `mode` above, by the
 * route of rtt_gram_normal with the collapse and its adjoint between the
 * FP64 forward and adjoint applies.  W^T W is an orthogonal projector, so no
 * eigenvalue exceeds the resolved arm's.  Same arguments as rtt_gram_normal
 * plus `mode`; synchronous.  Errors: RTT_EINVAL, RTT_ENOMEM, RTT_ECUDA.
 */
rtt_status rtt_gram_normal_mix(rtt_op op, int arm_mask, int mode, const double* Q_dev, int d,
                               double* G_dev, void* stream);

/*
 * rtt_eig_sym -- eigendecomposition of a symmetric n x n FP64 matrix on the
 * GPU (parallel cyclic Jacobi, round-robin ordering, relative off-diagonal
 * criterion), as used for the spectrum of the restricted Gram (Eq. 31).
 * A_dev is overwritten (its diagonal holds the eigenvalues); V_dev receives
 * the eigenvectors as columns (row-major n x n); evals_host receives the
 * unsorted eigenvalues; sweeps_host (optional) the sweep count.
 * Errors: RTT_EINVAL, RTT_ENOTCONVERGED (max_sweeps reached), RTT_ECUDA.
 */
rtt_status rtt_eig_sym(int n, double* A_dev, double* evals_host, double* V_dev, int max_sweeps,
                       int* sweeps_host, void* stream);

/*
 * rtt_eigvals_sym_batched -- eigenvalues only (ascending, evals_host: batch *
 * n) of `batch` consecutive symmetric n x n FP64 matrices in A_dev (row-major,
 * overwritten): Householder reduction to tridiagonal form and bisection with
 * Sturm counts, one CTA per matrix (the spectra of restricted Grams, Eq.
 * 31).  Absolute error of order n eps ||A||;
 * for eigenvalues that must be resolved relative to their own size near a
 * threshold use rtt_eig_sym (the rank audit does so automatically).
 * Synchronous.  Errors: RTT_EINVAL, RTT_ECUDA.
 */
rtt_status rtt_eigvals_sym_batched(int n, int batch, double* A_dev, double* evals_host,
                                   void* stream);

/* rtt_eig_sym on `batch` matrices at once (A_dev, V_dev: batch consecutive
   n x n blocks; evals_host: batch * n; sweeps_host: batch ints), one CTA per
   matrix (Eq. 31 for several Grams in one launch).  Errors as rtt_eig_sym,
   and RTT_EINVAL for batch < 1. */
rtt_status rtt_eig_sym_batched(int n, int batch, double* A_dev, double* evals_host, double* V_dev,
                               int max_sweeps, int* sweeps_host, void* stream);

/*
 * rtt_gemm_tn_f64 -- C = A^T B in FP64 accuracy on the tensor cores: the
 * contraction of the restricted Gram, G = Q^T (A^T A Q) (Eq. 21), and of the
 * TSVD projections (Sec. 9).  A: k x m, B: k x n, C: m x n, FP64 device
 * memory, row-major with row strides lda >= m, ldb >= n, ldc >= n.  Every
 * column of A and of B is scaled by a power of two and split exactly into
 * seven signed 7-bit integer digits (BF16); the 28 digit pairs whose weights
 * reach 2^-56 are multiplied by tcgen05.mma with FP32 accumulation over
 * windows of 128 k (exact: the sums stay below 2^22), and the windows are
 * added in 64-bit integers, so the result is deterministic and its error is
 * that of truncating each operand column to 49 bits below its largest entry
 * (about 2^-46 of sum_k |A_ki| |B_kj| scaled by the column maxima).
 * 1 <= k < 2^27.  Allocates its workspace (digit slices, 14 (m + n) k bytes)
 * and synchronises `stream`.
 * Errors: RTT_EINVAL, RTT_ENOMEM, RTT_ECUDA, RTT_ETIMEOUT (a bounded wait of
 * the kernel gave up).
 */
rtt_status rtt_gemm_tn_f64(int64_t k, int m, int n, const double* A_dev, int64_t lda,
                           const double* B_dev, int64_t ldb, double* C_dev, int64_t ldc,
                           void* stream);

/*
 * rtt_range_finder -- adaptive randomized range finder with an FP64
 * projected eigensolve for the spectrum of the restricted normal operator
 * H = Q^T A^T A Q of a class (Sec. 7-8, the spectra of the larger classes;
 * Eq. 31).  Q_dev: double [n_nodes][n_hats][d] (device); omega_host: the
 * caller's Gaussian draws, double [d][block * max_blocks] row-major (block
 * i = columns i*block .. i*block + block - 1).  Per block: Y = H Omega_i
 * (FP64 applies of A and A^T, contractions with Q by rtt_gemm_tn_f64), Y
 * made orthogonal to the basis found so far (twice) and orthonormal by
 * Householder QR with column pivoting (FP64, host; columns whose pivot is
 * below 1e-12 of Y's largest column norm dropped), then the Ritz values of H
 * on the whole basis (its Gram with H applied, Jacobi eigensolver).  Stops after a block that adds no Ritz value at or
 * above rho^2, once the basis has d vectors, or after max_blocks.  Ritz
 * values never exceed H's eigenvalues, so *rank_out (sigma >= rho, sigma =
 * sqrt of a Ritz value) never exceeds the operational rank, and equals it
 * once the basis spans the class.  sigma_out: host, capacity d, the
 * *n_sigma_out singular values descending; blocks_out (optional): blocks
 * used.  Synchronous.
 * Errors: RTT_EINVAL, RTT_ESTATE (row shard), RTT_ENOMEM, RTT_ECUDA,
 * RTT_ETIMEOUT (a bounded device wait of the contraction timed out),
 * RTT_ENOTCONVERGED (the eigensolver).
 */
rtt_status rtt_range_finder(rtt_op op, int arm_mask, const double* Q_dev, int d, int block,
                            int max_blocks, const double* omega_host, double rho,
                            double* sigma_out, int* n_sigma_out, int* rank_out, int* blocks_out,
                            void* stream);

/*
 * rtt_operational_rank -- operational rank of a restricted Gram from its
 * eigenvalues (Sec. 4.4 Eq. 31): sigma_i = sqrt(max(lambda_i, 0)) (the
 * whitening scale SNR_0 / s_ref is already in the Gram), rank = #{sigma_i >=
 * rho} (inclusive), margin = min_i |sigma_i - rho| / rho.  evals_host: n
 * eigenvalues in any order; sigma_out_host (optional, n doubles) receives the
 * sigma_i sorted descending; rank_out and margin_out: host scalars.
 * Errors: RTT_EINVAL (n < 1, null pointers, rho <= 0, non-finite
 * eigenvalue).
 */
rtt_status rtt_operational_rank(int n, const double* evals_host, double rho, int* rank_out,
                                double* margin_out, double* sigma_out_host);

/*
 * rtt_solve_ridge -- ridge / Tikhonov estimator (Sec. 9):
 * (A^T A + lambda I) x = A^T d, with A the whitened operator of the arm, for
 * n_rhs data columns and n_lambda values at once (output column
 * c = rhs * n_lambda + l).  data_dev: float [arm_rows][n_frames][n_rhs];
 * x_dev: float [n_nodes][n_hats][n_rhs * n_lambda] (overwritten; the
 * starting guess is 0).  Batched conjugate gradients with FP32 vectors and
 * applies, FP64 per-column dot products in a fixed order, and the residual
 * recomputed in FP64 every refresh_every iterations.  A column stops when
 * its recurrence residual falls below tol * ||A^T d||.  iters_out: host int
 * (iterations run); relres_out: host double [n_rhs * n_lambda], the final
 * FP64 relative residual of each column.  Synchronous.
 * Errors: RTT_EINVAL, RTT_ENOMEM, RTT_ECUDA, RTT_ENOTCONVERGED (max_iter
 * reached; x and relres_out still hold the last iterate's values).
 */
rtt_status rtt_solve_ridge(rtt_op op, int arm_mask, const float* data_dev, int n_rhs,
                           const double* lambdas_host, int n_lambda, int max_iter, double tol,
                           int refresh_every, float* x_dev, int* iters_out, double* relres_out,
                           void* stream);

/*
 * rtt_solve_tsvd -- truncated-SVD estimator in a representation class
 * (Sec. 9): x = Q V_r L_r^{-1} V_r^T Q^T A^T d, where (V, L) are the
 * eigenpairs of the restricted Gram G = P^T P (rtt_gram, rtt_eig_sym) sorted
 * by descending eigenvalue and r = rank (the paper truncates at the
 * operational rank).  Q_dev: double [n_nodes][n_hats][d]; V_dev: double
 * [d][d] row-major, eigenvectors as columns; evals_host: d doubles, the first
 * `rank` positive; data_dev: double [arm_rows][n_frames][n_rhs]; xhat_dev:
 * double [n_nodes][n_hats][n_rhs].  FP64; the plain GEMMs use cuBLAS.
 * Synchronous.  Errors: RTT_EINVAL, RTT_ENOMEM, RTT_ECUDA.
 */
rtt_status rtt_solve_tsvd(rtt_op op, int arm_mask, const double* Q_dev, int d, const double* V_dev,
                          const double* evals_host, int rank, const double* data_dev, int n_rhs,
                          double* xhat_dev, void* stream);

/* One (geometry, observation arm) record of the rank audit. */
typedef struct {
    int32_t arm_mask;
    int32_t rank;          /* operational rank #{sigma_i >= rho} (Eq. 31) */
    double margin;         /* min_i |sigma_i - rho| / rho: distance of the decision */
    double sigma_max;
    double sigma_min_pos;  /* smallest positive sigma (positive-support conditioning) */
    double s_ref;          /* Eq. 17 of the geometry */
    int32_t jacobi_sweeps;
    rtt_reach_result reach; /* anchor, L_anchor, T_reach, A_0,q, J_old */
    double seconds;        /* wall time of this record */
    double seconds_probe;  /* of which: age probes and reach */
    double seconds_gram;   /* of which: restricted Gram */
    double seconds_eig;    /* of which: share of the batched eigensolve */
} rtt_audit_record;

#define RTT_GRAM_DATA 0   /* G = P^T P over data samples (rtt_gram) */
#define RTT_GRAM_NORMAL 1 /* G = Q^T A^T A Q (rtt_gram_normal) */
#define RTT_GRAM_CLASS_S224 2 /* rtt_gram_class for the S224 class (Q_dev may be NULL) */
#define RTT_GRAM_CLASS_L224 3 /* rtt_gram_class for the L224 class (Q_dev may be NULL) */

/*
 * rtt_rank_audit -- the audit of Sec. 6.2-6.3 for n_ops geometries: for each
 * operator ops[g] with class Q_dev[g] (double [n_nodes][n_hats][d], e.g. the
 * S224 synthesis of Eq. 8) and each arm in arm_masks (e.g. direct 0x1 and
 * resolved 0x7): probe information on the n_ages ages_host (width h),
 * anchor-connected reach, the direct age boundary A_{0,quantile} (shared by
 * the arms of a geometry) and J_old (Eq. 35), then G = P^T P, P = scale A Q
 * (FP64; gram_mode RTT_GRAM_DATA uses rtt_gram, RTT_GRAM_NORMAL uses
 * rtt_gram_normal, RTT_GRAM_CLASS_S224 / _L224 use rtt_gram_class for that
 * class and d must be 224; where rtt_gram_class returns RTT_ESTATE the
 * normal-operator Gram of Q_dev[g] is taken instead, which then must not be
 * NULL), its spectrum (rtt_eigvals_sym_batched; a matrix with an eigenvalue
 * within 64 d eps max|lambda| of rho^2 is recomputed with the Jacobi
 * eigensolver) and the operational rank.  The class modes run as one batched
 * plan (rtt_audit_plan_*) unless a geometry has rows the class path does not
 * handle.
 * out: host array [n_ops][n_arms]; sigma_out (optional): host
 * [n_ops][n_arms][d], singular values descending.  Synchronous.
 */
rtt_status rtt_rank_audit(const rtt_op* ops, int n_ops, const double* const* Q_dev, int d,
                          const int* arm_masks, int n_arms, int n_ages, const double* ages_host,
                          double h, double quantile, int gram_mode, rtt_audit_record* out,
                          double* sigma_out, void* stream);

/*
 * Batched audit plan (Sec. 6.2-6.3, the audit of rtt_rank_audit for the
 * separable classes, one launch per stage over every (geometry, arm) job).
 * rtt_audit_plan_create: validates, computes each geometry's A_{0,quantile}
 * (Sec. 4.5), builds every geometry's class tables (factor tables, ray-space
 * values, per-row temporal blocks of Eq. 21's separable form) and allocates
 * every buffer of the run; synchronises `stream`.  class_kind:
 * RTT_CLASS_S224 or RTT_CLASS_L224 (d = 224).  Jobs are geometry-major:
 * record j = g n_arms + a.
 * rtt_audit_plan_run: enqueues the run on `stream` with no host
 * synchronisation and no allocation (capturable in a CUDA graph): the probes
 * of Eq. 10-12 and 29 of all jobs (FP32 pass; FP64 re-evaluation of the ages
 * within 1e-3 of rho^2, decided on the device), the class Grams of all jobs,
 * and their eigenvalues (tridiagonal reduction and bisection).
 * rtt_audit_plan_results: synchronises `stream` and fills out[n_ops * n_arms]
 * (and sigma_out [n_ops][n_arms][224], descending, if not NULL) with the
 * reach and J_old (Eq. 13, 30, 33-35) and the operational rank (Eq. 31); a
 * spectrum with an eigenvalue within 64 d eps max|lambda| of rho^2 is
 * recomputed by the Jacobi eigensolver first.  The stage times of the run
 * (CUDA events) are shared evenly by the records.
 * Errors: RTT_EINVAL (arguments, null operator), RTT_ESTATE (a row shard; a
 * geometry with rows the class path does not handle, create; results before
 * a run), RTT_ENOMEM, RTT_ECUDA.
 */
typedef struct rtt_audit_plan_s* rtt_audit_plan;
rtt_status rtt_audit_plan_create(const rtt_op* ops, int n_ops, const int* arm_masks, int n_arms,
                                 int n_ages, const double* ages_host, double h, double quantile,
                                 int class_kind, void* stream, rtt_audit_plan* out);
rtt_status rtt_audit_plan_run(rtt_audit_plan plan, void* stream);
rtt_status rtt_audit_plan_results(rtt_audit_plan plan, rtt_audit_record* out, double* sigma_out,
                                  void* stream);
rtt_status rtt_audit_plan_destroy(rtt_audit_plan plan);

/*
 * rtt_autotune -- choose the fastest kernel variants of the FP32 applies
 * (rtt_apply_A / rtt_apply_AT) of this operator for one batch size.  The
 * paper has no counterpart: this is a property of the GPU implementation.
 * Candidates: the forward with staged per-ray histories (corner rows loaded
 * by threads or by TMA tensor copies) or with one hat per lane and warp
 * shuffles (the latter only when a frame step is 1/2, 1/4 or 1/8 of a hat
 * step), each with a few batch widths and frames per lane; the adjoint's
 * cell kernel with frames staged by per-lane copies, or by TMA tensor copies
 * with 32-hat or 64-hat items.  Each candidate runs once untimed and three
 * times between CUDA events on `stream`, on zero-filled inputs of the arm's
 * shape (timing does not depend on values).  The fastest is recorded in the
 * operator for `batch` (up to 8 batch sizes per operator; later applies of
 * that batch size use it).  Every variant sums each output in the same order
 * with the same fused multiply-adds, so tuning never changes a result bit.
 * Allocates temporaries (x and y of the batch, cudaMalloc/cudaFree) and
 * synchronises the stream: call it before any graph capture, not
 * concurrently with applies on the same operator.
 * out: host struct (below).  Errors: RTT_EINVAL (batch outside 1..4096, bad
 * arm), RTT_ENOMEM, RTT_ECUDA.
 */
typedef struct {
    int32_t batch;
    int32_t fwd_kernel;   /* 1 staged, 2 lane-per-hat, 3 staged with TMA corner copies,
                             4 staged with pipelined bulk corner copies, 5 periodic
                             staged with the whole batch in one chunk, 6 the same with
                             its table loads one task ahead, 7 periodic quad-lane, 8 the
                             same with its table loads one task ahead, 9 quad-lane with
                             the corner slabs staged one ray ahead */
    int32_t fwd_bc;       /* batch entries per forward task */
    int32_t fwd_frames_per_lane;
    int32_t fwd_staging;  /* staged forward: x items in flight per lane */
    int32_t adj_kernel;   /* adjoint: 1 general, 2 periodic staged by per-lane copies,
                             3 TMA with 32-hat items, 4 TMA with 64-hat items */
    float fwd_ms, adj_ms;           /* chosen variants, ms per apply */
    float fwd_ms_rule, adj_ms_rule; /* the untuned default rule, ms per apply */
    int32_t candidates;             /* configurations timed */
    int32_t fwd_order;    /* forward task rows: 0 (order, pixel), 1 source-cell order */
    int32_t fwd_cols;     /* forward column passes (0: all columns at once) */
    int32_t adj_cols;     /* adjoint columns per pass (0: 32 in FP32, 64 at batches of whole
                             64-column passes) */
} rtt_tune_result;

rtt_status rtt_autotune(rtt_op op, int batch, int arm_mask, void* stream, rtt_tune_result* out);

/* A kernel variant of the FP32 applies (the same choices rtt_autotune makes). */
typedef struct {
    int32_t fwd_kernel;   /* 1 staged, 2 lane-per-hat (periodic cadences; else staged),
                             3 staged with TMA corner copies (batch a multiple of 4;
                             else staged), 4 staged with bulk corner copies pipelined
                             two rays ahead (batch 4 or 8 as one chunk; else staged),
                             5 periodic staged with the whole batch in one chunk and
                             32-bit hat arithmetic (periodic cadences, batch 4 or 8;
                             else staged), 6 kernel 5 with each task's table loads
                             issued during the task before it, 7 periodic quad-lane:
                             fwd_bc / 4 lanes share a frame, each holding 4 of its
                             columns, so every store instruction writes 512 contiguous
                             bytes (periodic cadences, chunks of 4..64 columns dividing
                             the batch; at batches of 1 or 2 columns a lane holds 4 / B
                             consecutive frames instead; else staged), 8 kernel 7 with
                             each task's table
                             loads issued during the task before it, 9 kernel 7 with each
                             ray's corner rows of x copied into shared memory (per-lane
                             asynchronous copies) during the ray before it */
    int32_t fwd_bc;       /* batch entries per forward task: 1, 2, 4, 8, 16 or 32; 64 for
                             fwd_kernel 7 to 9 */
    int32_t fwd_half;     /* staged forward: 1 = half the frames per lane */
    int32_t adj_kernel;   /* adjoint: 1 general (any cadence, batch and precision; frames
                             staged by per-lane copies), 2 periodic (a frame step of 1/2,
                             1/4 or 1/8 hat step; any batch, in 8- or 4-column chunks;
                             frames staged by per-lane copies), 3 frames staged by TMA
                             tensor copies with 32-hat items, 4 the same with 64-hat items
                             (TMA: the whole batch of 4, 8 or 16 entries in one chunk with
                             whole frames per 128-byte line; at batches of whole 32-column
                             passes both run the TMA kernel of 32- or (batches of whole
                             64-column passes) 64-column passes, 16- or 8-hat items with
                             two or four lanes per hat; at batches of 1 or 2 columns both
                             run the direct-load kernel, 32- or 64-hat items); where the call
                             does not allow the choice, the next one down runs */
    int32_t fwd_staging;  /* staged forward: x items in flight per lane, 1, 2 or 3
                             (0 = 2; other values than 2 only at 4 or 8 entries) */
    int32_t fwd_order;    /* forward task rows: 0 in (order, pixel) order, 1 in source-cell
                             order (within each order, by the Morton index of the row's
                             first ray's cell: rows that read the same x nodes run
                             close together) */
    int32_t fwd_cols;     /* periodic forward (fwd_kernel 5, 6): 0 = all columns in one
                             launch, or a multiple of 4 dividing the batch = the whole
                             operator for that many columns at a time (bounds x's and
                             y's working set for large batches); 0..64 */
    int32_t adj_cols;     /* adjoint columns per pass (0 = 32, or 64 at batches of whole
                             64-column passes; else 4..32, a multiple of 4): the partial
                             records hold one pass */
} rtt_variant;

/*
 * rtt_set_variant / rtt_get_variant -- pin (or, with v == NULL, reset to the
 * default rule) the kernel variant used by FP32 applies of `batch` columns,
 * or read the one in force.  For manual tuning and for tests that run every
 * variant; results are the same bits for every variant.  Not thread-safe
 * against concurrent applies on the same operator.  The paper has no
 * counterpart (a property of this GPU implementation).  Errors: RTT_EINVAL.
 */
rtt_status rtt_set_variant(rtt_op op, int batch, const rtt_variant* v);
rtt_status rtt_get_variant(rtt_op op, int batch, rtt_variant* out);

/*
 * rtt_destroy -- free the operator and every device buffer it owns (tables,
 * index arrays, scratch).  Work queued on a stream that uses `op` must have
 * completed.  A null op is ignored.  Library plumbing: the paper has no
 * counterpart.  Never fails.
 */
void rtt_destroy(rtt_op op);

#ifdef __cplusplus
}
#endif

#endif /* RTT_H */
