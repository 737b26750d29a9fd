/*
 * dcrf.h -- C ABI of the GB300 dense-CRF filtering hot path.
 *
 * Efficient Continuous Relaxations for Dense CRF (Desmaison, Bunel, Kohli,
 * Torr, Kumar; arXiv 1608.06192).  The library computes, on one GPU, the dense
 * Gaussian pairwise product sum_b K(f_a, f_b) y_b over all label channels with
 * a permutohedral lattice (Section 3, "Filter-based Method", Eq. 6), and the
 * three solvers built on it: Frank-Wolfe on the convex QP relaxation (Section
 * 4, Algorithm 1, Appendix B), CCCP on the generic DC relaxation (Section 5.1,
 * Algorithm 2) and the LP relaxation's subgradient by sort + divide and
 * conquer (Section 6, Eq. 19-20, Appendix E) with projected subgradient steps
 * (Algorithm 3).
 *
 * Conventions for every entry point:
 *  - Pointers documented "device" must point to GPU memory owned by the
 *    caller (for example torch tensors), contiguous, row-major; "host"
 *    pointers are CPU memory.  The library never frees caller memory.
 *  - Pixels of a batch are concatenated: image b owns rows
 *    offsets[b] .. offsets[b+1]-1.  A single image is a batch of one.
 *  - Per-pixel label arrays are [N][L] float32, label-contiguous.
 *  - Calls are asynchronous on the given stream unless stated otherwise; the
 *    returned status covers argument checks and launch errors.  Errors found
 *    on the device (hash table full, key out of range, non-finite values,
 *    a bounded wait that expired) are recorded in a device status word of the
 *    lattice and returned by the next call that synchronises
 *    (dcrf_lattice_build, dcrf_lattice_status, and solver calls that copy
 *    records to the host).
 *  - No entry point launches work on a stream other than the one given.
 */
#ifndef DCRF_H
#define DCRF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *dcrf_stream;       /* a cudaStream_t; NULL = legacy default stream */
typedef struct dcrf_lattice_s *dcrf_lattice;   /* opaque, owned by the library */

typedef enum {
    DCRF_OK = 0,
    DCRF_E_INVAL = -1,       /* bad argument: null pointer, size, dimension, shapes that disagree */
    DCRF_E_NOMEM = -2,       /* device allocation failed */
    DCRF_E_CUDA = -3,        /* a CUDA runtime call or launch failed */
    DCRF_E_TABLE_FULL = -4,  /* lattice hash table ran out of slots (bounded probing) */
    DCRF_E_KEY_RANGE = -5,   /* a lattice coordinate does not fit the packed key */
    DCRF_E_TIMEOUT = -6,     /* a bounded device-side wait gave up */
    DCRF_E_NONFINITE = -7,   /* NaN or Inf met in inputs or a reduction */
    DCRF_E_SCRATCH = -8      /* the request does not fit dcrf_filter_static's fixed scratch */
} dcrf_status;

typedef enum {
    DCRF_STORAGE_F32 = 0,    /* lattice values stored in float32 */
    DCRF_STORAGE_F16 = 1     /* lattice values stored in float16, accumulated in float32 */
} dcrf_storage;

/* One Frank-Wolfe iteration of one image (Algorithm 1; Appendix B). */
typedef struct {
    double energy;   /* S_cvx(y^t) of Eq. 10 (or the CCCP inner objective) before the step */
    double gap;      /* <g, y^t - s>, g = (phi - d) + 2 (Psi + D) y^t  (Eq. 12, Eq. 14) */
    double alpha;    /* step taken, the minimiser over [0,1] of A a^2 + B a */
    double A;        /* (s - y)^T (Psi + D) (s - y) */
    double B;        /* derivative of the evaluated quadratic at a = 0 */
} dcrf_fw_record;

const char *dcrf_status_string(int status);
int dcrf_version(void);

/*
 * Step a1 -- features of Appendix G (kernel form of Eq. 4).
 * rgb: device [N][3] float32, the images of the batch concatenated, each
 *   row-major (pixel a = y*W + x).  widths, heights: host [batch]; an image
 *   may be empty (a width or height of 0).
 * f_bil: device [N][5] = (x/theta_alpha, y/theta_alpha, rgb/theta_beta).
 * f_sp:  device [N][2] = (x, y)/theta_gamma.  Either output may be NULL.
 * Each value is one correctly rounded float32 division.
 */
dcrf_status dcrf_features(const float *rgb, const int32_t *widths, const int32_t *heights, int batch,
                          float theta_alpha, float theta_beta, float theta_gamma,
                          float *f_bil, float *f_sp, dcrf_stream stream);

/*
 * Step a2 -- permutohedral lattice of one Gaussian kernel (Section 3 and
 * Appendix A of the paper, which cites Adams et al. for the method).
 * features: device [N][d] float32, already divided by the kernel widths, so
 *   that the kernel is exp(-|f_a - f_b|^2 / 2).  1 <= d <= 8.
 * offsets: host [batch+1], offsets[0] = 0, offsets[batch] = N; each image
 *   gets its own lattice (points of different images never interact).
 * On success *out owns the device arrays of the lattice: enclosing simplex
 * of every point (vertex ids and barycentric weights), vertex keys, blur
 * neighbours and K~1 (the filtered ones vector).  The build synchronises the
 * stream once (to read the vertex count) and returns DCRF_E_TABLE_FULL or
 * DCRF_E_KEY_RANGE when the device reported it; *out is then NULL.
 * A lattice is immutable after the build and may be read from any stream.
 * Its arrays come from the library's device pool (see dcrf_pool_trim) of the
 * stream's device; dcrf_lattice_destroy synchronises the device and returns
 * them to that pool.
 */
dcrf_status dcrf_lattice_build(const float *features, int64_t n, int d, dcrf_stream stream,
                               dcrf_lattice *out);
dcrf_status dcrf_lattice_build_batch(const float *features, const int64_t *offsets, int batch, int d,
                                     dcrf_stream stream, dcrf_lattice *out);
dcrf_status dcrf_lattice_destroy(dcrf_lattice lat);

/* Sizes: n points, d features, m vertices, batch images (any output may be NULL). */
dcrf_status dcrf_lattice_info(dcrf_lattice lat, int64_t *n, int *d, int64_t *m, int *batch);

/* host [batch+1]: vertex range of each image. */
dcrf_status dcrf_lattice_vertex_offsets(dcrf_lattice lat, int64_t *offsets);

/* Reads and clears the device status word (synchronises the stream). */
dcrf_status dcrf_lattice_status(dcrf_lattice lat, dcrf_stream stream);

/*
 * Copies the lattice structure into caller buffers (device; any may be NULL):
 * keys [m][d] int32 (vertex coordinates 0..d-1; coordinate d is minus their
 * sum), point_vertex [n][d+1] int32, point_weight [n][d+1] float32,
 * neighbours [m][d+1][2] int32 (vertex id of v - w_j, v + w_j or -1).
 */
dcrf_status dcrf_lattice_export(dcrf_lattice lat, int32_t *keys, int32_t *point_vertex,
                                float *point_weight, int32_t *neighbours, dcrf_stream stream);

/*
 * Check mode for the tables the kernels index with (no counterpart in the
 * paper).  point_vertex [n][d+1] int32, point_weight [n][d+1] float32 and
 * neighbours [m][d+1][2] int32 are device arrays laid out as
 * dcrf_lattice_export writes them; point_offsets and vertex_offsets are host
 * [batch+1] (points and vertices of each image).  A table passes when every
 * corner's vertex is -1 or a vertex of the point's own image, every weight is
 * finite in [0, 1] and each point's weights sum to one within 1e-5, and every
 * blur neighbour is -1 or a vertex of the same image.  Synchronises; returns
 * DCRF_E_INVAL when an entry fails (bad_entries, host, may be NULL, receives
 * how many) or when the sizes disagree.  dcrf_lattice_validate runs it on a
 * lattice's own tables.
 */
dcrf_status dcrf_check_lattice_tables(const int32_t *point_vertex, const float *point_weight, int64_t n, int d,
                                      const int32_t *neighbours, int64_t m, const int64_t *point_offsets,
                                      const int64_t *vertex_offsets, int batch, int64_t *bad_entries,
                                      dcrf_stream stream);
dcrf_status dcrf_lattice_validate(dcrf_lattice lat, int64_t *bad_entries, dcrf_stream stream);

/*
 * Eq. 6 through the lattice: out = K~ Y, K~ = s0 S^T B_d ... B_0 S, i.e.
 * splat, d+1 axis blurs [1/4, 1/2, 1/4] (axis order 0..d), slice; not
 * normalised (Appendix A).  Y, out: device [N][L] float32 (out may not alias
 * Y), 1 <= L <= 64.  storage selects float32 or float16 lattice values.
 */
dcrf_status dcrf_filter(dcrf_lattice lat, const float *Y, int L, float *out, int storage,
                        dcrf_stream stream);

/*
 * dcrf_filter without any device allocation.  No counterpart in the paper:
 * it exists for callers that cannot allocate device memory when they filter
 * (for example while capturing a stream under a mode that forbids
 * allocation, or real-time code with a fixed memory budget).  Same result and
 * arguments as dcrf_filter; the splat and blur buffers live in one
 * file-scope device array of dcrf_filter_static_capacity() bytes (16 MiB),
 * which every GPU that loads the library holds until the process exits.
 * Requests with lattice vertices * round4(L) * (4 + 2 * value size) bytes
 * (each part rounded up to 256) above that size return DCRF_E_SCRATCH.
 * The array's device address is looked up once per device (with that device
 * current) by dcrf_lattice_build, or else by the first dcrf_filter_static
 * call on the stream's device; when a call has to do it, make that call
 * before any stream capture.  All
 * calls share the array and it keeps the last call's contents (the splat
 * buffer is cleared on entry): calls that overlap on the GPU race, so
 * serialise them.
 */
dcrf_status dcrf_filter_static(dcrf_lattice lat, const float *Y, int L, float *out, int storage,
                               dcrf_stream stream);
size_t dcrf_filter_static_capacity(void);

/* Adjoint K~^T U: the same chain with the blur axes in reverse order. */
dcrf_status dcrf_filter_adjoint(dcrf_lattice lat, const float *U, int L, float *out, int storage,
                                dcrf_stream stream);

/*
 * Frank-Wolfe on the convex QP relaxation S_cvx (Eq. 10; Algorithm 1 with the
 * closed-form step and product reuse of Appendix B).
 * unaries: device [N][L] phi.  lattices: host [n_kernels] handles over the
 *   same points and batch; weights: host [n_kernels] w_m >= 0.
 * compat: host [L][L] label compatibility mu, or NULL for Potts [i != j].
 * Y: device [N][L]; on entry y^0 (rows on the simplex), on exit y^iters.
 * The rows of y^0 are checked on the device (non-negative, summing to one
 * within 1e-5); a row that is not is reported as DCRF_E_INVAL in the status
 * word, returned here when records are asked for.
 * records: host [iters][batch] or NULL; when given, the call synchronises.
 * Pairwise operator: Psi = mu (x) (sum_m w_m K~_m - (sum_m w_m) I) (Eq. 7),
 * d_a(i) = (sum_j |mu_ij|) max(0, (K~1)_a - sum_m w_m) (Eq. 11).
 * One filter-equivalent per iteration; the step uses the exact derivative of
 * the evaluated quadratic and is clipped to [0, 1].
 */
dcrf_status dcrf_qp_fw(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                       int n_kernels, const float *compat, int L, int iters, float *Y,
                       dcrf_fw_record *records, int storage, dcrf_stream stream);

/*
 * dcrf_qp_fw that also returns the solver's decisions: s_trace, device uint8
 * [iters][N], receives in row t the conditional gradient s^t = argmin_i g_a(i)
 * of iteration t for every pixel (Eq. 14; row 0 is the argmin at y^0).  The
 * rows make a run reproducible outside the library: replaying them through
 * Algorithm 1 with the closed-form step of Appendix B retraces y^t exactly up
 * to rounding, also where an argmin is within rounding of a tie.  s_trace may
 * be NULL (then this is dcrf_qp_fw).  Costs one copy of N bytes per iteration.
 */
dcrf_status dcrf_qp_fw_trace(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                             int n_kernels, const float *compat, int L, int iters, float *Y,
                             dcrf_fw_record *records, uint8_t *s_trace, int storage, dcrf_stream stream);

/*
 * The whole QP path from host memory in one call: features (Eq. 4), the
 * bilateral (d = 5) and spatial (d = 2) lattices, `iters` Frank-Wolfe
 * iterations as dcrf_qp_fw, and y back to the host.
 * rgb: host [N][3]; unaries: host [N][L]; Y0: host [N][L] (rows on the
 * simplex); Y: host [N][L] output (may be Y0).  widths, heights: host
 * [batch], N = sum of widths x heights.  thetas as dcrf_features; weights:
 * host [2] (bilateral, spatial); compat, records and storage as dcrf_qp_fw.
 * Device memory is taken from the stream-ordered allocator and released
 * before the return.  The unaries and y0 upload on a second stream while the
 * lattices are built; with page-locked host memory (cudaHostAlloc,
 * cudaHostRegister) that upload overlaps the builds, with pageable memory it
 * is synchronous.  Synchronises before returning; errors as the steps.
 */
dcrf_status dcrf_qp_fw_host(const float *rgb, const float *unaries, const float *Y0, float *Y,
                            const int32_t *widths, const int32_t *heights, int batch, int L, float theta_alpha,
                            float theta_beta, float theta_gamma, const float *weights, const float *compat,
                            int iters, dcrf_fw_record *records, int storage, dcrf_stream stream);

/*
 * Reverse mode through `iters` unrolled Frank-Wolfe iterations (the
 * differentiation pattern of this library; the paper names learning through
 * its solvers as future work in its discussion).  Given dYT = dLoss/dy^T for
 * y^T = dcrf_qp_fw(phi, w, y^0), returns dphi (device [N][L]), dY0 (device
 * [N][L] or NULL) and dweights (host [n_kernels], summed over the batch, or
 * NULL; when given the call synchronises).  The forward pass is recomputed
 * from Y0 with float32 lattice values, checkpointing y^t and s^t of every
 * iteration.  s^t is piecewise constant and alpha is constant where it is
 * clipped to [0, 1]; elsewhere alpha = -B/(2A) is differentiated exactly,
 * with Op^T applied through dcrf_filter_adjoint's reverse blur.
 * s_tape: device uint8 [iters][N] or NULL: the recomputed forward's
 * decisions s^t (as dcrf_qp_fw_trace), i.e. the smooth piece of the unrolled
 * map whose derivative was taken.
 */
dcrf_status dcrf_qp_fw_backward(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                                int n_kernels, const float *compat, int L, int iters, const float *Y0,
                                const float *dYT, float *dphi, float *dY0, double *dweights,
                                uint8_t *s_tape, dcrf_stream stream);

/*
 * CCCP on the generic DC relaxation (Section 5.1, Algorithm 2): outer steps
 * linearise q(y) = y^T D y at y^t and run `inner` Frank-Wolfe iterations on
 * phi^T y + y^T (Psi + D) y - 2 (d o y^t)^T y, warm-started at y^t.
 * qp_energy: host [outer+1][batch] or NULL: S_QP(y) = phi^T y + y^T Psi y
 * (Eq. 8) at the start and after every outer step (synchronises).
 */
dcrf_status dcrf_dc_cccp(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                         int n_kernels, const float *compat, int L, int outer, int inner, float *Y,
                         double *qp_energy, int storage, dcrf_stream stream);
/* dcrf_dc_cccp that also returns the decisions: s_trace, device uint8
 * [outer * inner][N], row o * inner + i = the conditional gradient of inner
 * Frank-Wolfe iteration i of outer step o (as dcrf_qp_fw_trace); may be NULL. */
dcrf_status dcrf_dc_cccp_trace(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                               int n_kernels, const float *compat, int L, int outer, int inner, float *Y,
                               double *qp_energy, uint8_t *s_trace, int storage, dcrf_stream stream);

/*
 * CCCP on the DC relaxation for negative semi-definite compatibilities
 * (Section 5.2, Appendix C).  S_QP(y) = [phi^T y - sum_w y^T (mu (x) I) y]
 * + [y^T (mu (x) K~) y]; each of the `outer` steps filters y^t once (one
 * splat, the forward and the reverse blur, one slice: F = K~ y + K~^T y) and
 * solves the per-pixel problems min lin_a^T y_a - sum_w y_a^T mu y_a over the
 * simplex with lin_a = phi_a + mu F_a: for Potts (compat NULL or 1 - I) the
 * Euclidean projection of -lin_a / (2 sum_w); otherwise `inner` Frank-Wolfe
 * steps per pixel with the exact step (compat must be symmetric; it should be
 * negative semi-definite on zero-sum vectors for CCCP's monotone decrease).
 * Y: device [N][L] on the simplex, updated in place.  qp_energy: host
 * [outer+1][batch] or NULL: S_QP at the start and after every outer step
 * (synchronises).  Errors: DCRF_E_INVAL for a bad argument, an asymmetric
 * compat or sum_w = 0; DCRF_E_NONFINITE for non-finite data.
 */
dcrf_status dcrf_dc_neg(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                        int n_kernels, const float *compat, int L, int outer, int inner, float *Y,
                        double *qp_energy, int storage, dcrf_stream stream);

/*
 * Parallel mean field, the baseline the paper compares with (Section 1,
 * Section 6.2: MF, and MF5 = 5 iterations), for P(x) proportional to
 * exp(-E(x)) with E of Eq. 1 (ordered pairs):
 *   Q <- softmax_rows(-phi - (Psi + Psi^T) Q),  Psi = mu (x) (K~ - sum_w I),
 * one filter per iteration (one splat, the forward and the reverse blur, one
 * slice).  Q: device [N][L], rows on the simplex (e.g. softmax(-phi)), updated
 * in place.  qp_energy: host [iters+1][batch] or NULL: S_QP(Q) = phi^T Q +
 * Q^T Psi Q before every update and at the end (synchronises).  compat must
 * be symmetric (NULL: Potts).
 */
dcrf_status dcrf_mean_field(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                            int n_kernels, const float *compat, int L, int iters, float *Q,
                            double *qp_energy, int storage, dcrf_stream stream);

/*
 * Rounding of a relaxed solution: labels[a] = argmax_i Y[a][i] (lowest label
 * on ties), int32 device [N]; onehot: device [N][L] or NULL.  Asynchronous.
 */
dcrf_status dcrf_round(const float *Y, int64_t n, int L, int32_t *labels, float *onehot, dcrf_stream stream);

/*
 * Kleinberg-Tardos rounding of an LP point (end of Section 5: the rounding
 * that gives the LP its factor 2 for the Potts model).  Phase t gives label
 * phase_labels[t] to every unlabelled pixel a with
 * Y[a][phase_labels[t]] > phase_thresholds[t] (FP32 comparison).  The random
 * draws are inputs: host arrays [n_phases] with labels uniform in [0, L) and
 * thresholds uniform in [0, 1), copied before the call returns.  Y: device
 * FP32 [N][L] (rows on the simplex); labels: device int32 [N], written with
 * the first label each pixel gets, -1 where no phase labelled it; with
 * resume != 0 its entries >= 0 are kept as they are and only the others are
 * processed (a run continued with further phases).  With T phases a pixel
 * stays unlabelled with probability (1 - 1/L)^T.  unassigned: host, the
 * number of pixels left at -1 (synchronises), or NULL (asynchronous).
 * DCRF_E_INVAL for a phase label outside [0, L) or a threshold outside [0, 1).
 */
dcrf_status dcrf_round_kt(const float *Y, int64_t n, int L, int n_phases, const int32_t *phase_labels,
                          const float *phase_thresholds, int resume, int32_t *labels, int64_t *unassigned,
                          dcrf_stream stream);

/*
 * Energy of a labelling, Eq. 1 (ordered pairs, pixel operator through the
 * lattices): E(x) = S_QP at the one-hot rows of x.  labels: device int32 [N]
 * in [0, L) (else DCRF_E_INVAL); energy: host [batch] (synchronises).
 * compat must be symmetric (NULL: Potts).
 */
dcrf_status dcrf_labelling_energy(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                                  int n_kernels, const float *compat, int L, const int32_t *labels,
                                  double *energy, int storage, dcrf_stream stream);

/*
 * LP relaxation subgradient (Eq. 18-20, Appendix D-E), Potts model.
 * For every label i the pixels are sorted by descending y_a(i) (ties by
 * ascending pixel index); the upper sums U_c = sum_{b after c} K~_cb come
 * from the divide and conquer of Appendix E with power-of-two splits, where
 * each sub-problem uses the lattice restricted to its own points; then
 * G = phi + 2U - c with c_a = (K~1)_a - sum_m w_m.
 * unaries, Y: device [N][L]; G: device [N][L] output.
 * energy: host [batch] or NULL: S_LP(y) = <y, G> (synchronises).
 */
dcrf_status dcrf_lp_subgrad(const float *unaries, const float *Y, const dcrf_lattice *lattices,
                            const float *weights, int n_kernels, int L, float *G, double *energy,
                            dcrf_stream stream);

/*
 * Projected subgradient on the LP (Algorithm 3): y <- Proj_M(y - beta_t G),
 * beta_t = beta0 / (1 + t).  beta0 <= 0 selects, per image,
 * beta0 = 0.1 / max_{a,i} |G0_a(i) - mean_i G0_a(i)|.
 * Y: device [N][L], in: y^0, out: the iterate with the lowest S_LP seen.
 * energies: host [steps+1][batch] or NULL (synchronises).
 */
dcrf_status dcrf_lp_solve(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                          int n_kernels, int L, int steps, double beta0, float *Y, double *energies,
                          dcrf_stream stream);

/*
 * The LP for a tree (r-HST) label metric, Appendix F: the pairwise term
 * sum_T c_T sum_{a, b != a} K_ab |y_a(T) - y_b(T)| / 2 over the given
 * subtrees T, with y_a(T) = sum_{i in L(T)} y_a(i).  Every subtree column is
 * sorted (descending, ties by pixel index) and summed by the same divide and
 * conquer, and G_a(k) = phi_a(k) + sum_{T containing k} c_T (2 U_T(a) - c_a).
 * subtree_labels: host [n_subtrees] bit masks of L(T) (bit i = label i, L <= 64,
 * non-empty); subtree_weights: host [n_subtrees] c_T >= 0 (the length of the
 * edge above T).  The Potts model is the tree of single labels with c_T = 1.
 * Otherwise as dcrf_lp_subgrad (energy = <y, G>, the tree LP objective) and
 * dcrf_lp_solve.  DCRF_E_INVAL for an empty or out-of-range mask or a
 * negative or non-finite weight.
 */
dcrf_status dcrf_lp_subgrad_tree(const float *unaries, const float *Y, const dcrf_lattice *lattices,
                                 const float *weights, int n_kernels, int L, int n_subtrees,
                                 const uint64_t *subtree_labels, const float *subtree_weights, float *G,
                                 double *energy, dcrf_stream stream);
dcrf_status dcrf_lp_solve_tree(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                               int n_kernels, int L, int n_subtrees, const uint64_t *subtree_labels,
                               const float *subtree_weights, int steps, double beta0, float *Y,
                               double *energies, dcrf_stream stream);

/*
 * Device scratch: every call takes its temporary device memory from a
 * stream-ordered pool that the library keeps per device and that holds on to
 * memory between calls (DCRF_POOL=default in the environment uses the
 * device's default pool instead).  dcrf_pool_trim returns the pools' unused
 * memory to the driver; call it once the streams that ran library calls are
 * synchronised.
 */
dcrf_status dcrf_pool_trim(void);

/*
 * Measurement hooks (no counterpart in the paper): when enabled, every
 * kernel launch of the library is bracketed by CUDA events on its own stream
 * and solvers launch without internal graphs.  dcrf_profile_read
 * synchronises on the recorded events and fills up to `capacity` rows of
 * (kernel name, launches, summed milliseconds); it returns the row count.
 * names receive pointers to static strings.
 */
dcrf_status dcrf_profile_enable(int on);
dcrf_status dcrf_profile_reset(void);
int dcrf_profile_read(const char **names, int64_t *launches, double *ms, int capacity);

/*
 * Self-test of the bounded device-side wait (no counterpart in the paper).
 * The pixel pass of the Frank-Wolfe solver waits for its tile copies on an
 * mbarrier with a bounded number of polls and flags DCRF_E_TIMEOUT when they
 * run out instead of hanging.  This launches one block that polls an
 * mbarrier `polls` times (1 <= polls <= 2^26): with never_complete != 0 the
 * barrier waits for bytes that nothing sends (no copy is in flight), so the
 * wait runs out and DCRF_E_TIMEOUT lands in lat's status word (read it with
 * dcrf_lattice_status); with never_complete == 0 it completes at once.
 * Asynchronous; the context stays usable either way.
 */
dcrf_status dcrf_selftest_bounded_wait(dcrf_lattice lat, int64_t polls, int never_complete, dcrf_stream stream);

/* Euclidean projection of every row of V [N][L] onto the simplex (device). */
dcrf_status dcrf_simplex_project(const float *V, int64_t n, int L, float *Y, dcrf_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* DCRF_H */
