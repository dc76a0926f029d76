/*
 * vie.h - C ABI of the GB300 preconditioned periodic volume-integral-equation solver.
 *
 * Method: He, Gu, Sha & Chen, "Efficient volumetric method of moments for
 * modeling plasmonic thin-film solar cells with periodic structures"
 * (arXiv:1809.05334).  One a x b unit cell of a periodic thin-film stack is
 * meshed with tetrahedra; the flux density D is expanded in SWG functions
 * (Sec. 2.1), the Galerkin impedance matrix of Eq. (2) is filled with the 2D
 * periodic Green's function of Eq. (3)-(4), evaluated by Ewald's method
 * (Sec. 2.2), the system is solved by GMRES with the domain-wise diagonal
 * block preconditioner of Eq. (5)-(6) (Sec. 2.3), and the absorbed fraction
 * of Eq. (7) is returned per material domain.
 *
 * Conventions
 *  - Lengths in nm.  Permittivities use the physics sign (Im eps > 0 is lossy);
 *    the library works internally in the exp(j w t) convention of the paper.
 *  - Unknown n is the normal flux of D across face n divided by eps0.  Faces
 *    are numbered in order of first appearance scanning tetrahedra t = 0.. and
 *    local faces i = 0..3 (face i is opposite vertex i); T+ of an interior face
 *    is the lower-numbered tetrahedron; a pair of lateral faces on x=0/x=a
 *    (y=0/y=b) is one Bloch-periodic unknown with T+ on the x=0 (y=0) wall.
 *  - Complex numbers are interleaved (re, im) doubles.
 *  - All entry points are host functions.  Pointers are host pointers unless
 *    the argument says "device".  Inputs are copied; the caller keeps
 *    ownership of every buffer it passes.  Nothing is retained after return
 *    except inside the opaque context.
 *  - Errors are returned as negative vie_status codes; no exception crosses
 *    the ABI.  Positive codes mean a result with a warning.  vie_last_error()
 *    gives a one-line description of the last failure on a context.
 *  - A context is not thread safe; use one context per host thread.
 */
#ifndef VIE_H
#define VIE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VIE_MAX_DOMAINS 8

typedef struct vie_ctx vie_ctx;

typedef enum {
    VIE_OK = 0,
    VIE_NOT_CONVERGED = 1,      /* result returned, residual above tolerance        */
    VIE_PENDING = 2,            /* vie_server_poll: the request has not finished     */
    VIE_EINVAL = -1,            /* bad argument                                      */
    VIE_ENOMEM = -2,            /* device allocation failed                          */
    VIE_ECUDA = -3,             /* CUDA runtime / launch error                       */
    VIE_RAYLEIGH_ANOMALY = -4,  /* a Floquet mode is at grazing: g_p is singular     */
    VIE_DEVICE_TIMEOUT = -5,    /* a bounded wait inside a device kernel ran out (the
                                   kernel gave up and returned; the context stays
                                   usable, the solve has no result)                 */
    VIE_BAD_MESH = -6,          /* inverted tetrahedron or unmatched periodic walls  */
    VIE_CANCELLED = -7,         /* the request was cancelled (vie_server_cancel)     */
    VIE_BREAKDOWN = -8          /* zero or non-finite pivot while inverting a domain
                                   block of Eq. (6) (no pivoting): the preconditioner
                                   does not exist, the solve has no result; rerun
                                   with use_precond = 0                              */
} vie_status;

typedef enum {
    VIE_FP64 = 0,   /* Z, Krylov vectors and products in FP64                        */
    VIE_FP32 = 1,   /* Z stored in FP32 (near-singular integrals in FP64), FP32
                       GMRES inside FP64-residual iterative refinement           */
    VIE_FP16 = 2,   /* as VIE_FP32, and the GMRES products of every refinement
                       sweep read a second copy of Z in FP16 (one power-of-two
                       scale for the matrix, FP32 accumulation); the FP64
                       residual of each sweep still reads the FP32 Z, so the
                       converged answer is that of the FP32 Z                   */
    VIE_BF16 = 3    /* as VIE_FP16 with the second copy in BF16 (no scale)        */
} vie_precision;

typedef struct {
    int32_t precision;     /* vie_precision                                        */
    int32_t use_precond;   /* 1: diagonal-block preconditioner of Eq. (6); 0: none  */
    int32_t restart;       /* GMRES restart length (default 100)                   */
    int32_t max_iter;      /* total GMRES iterations over all restarts (default 1000)*/
    double  tol;           /* target FP64 relative residual ||b - Z x|| / ||b||     */
    double  inner_tol;     /* relative reduction of the preconditioned residual at
                              which a refinement sweep's inner GMRES stops (never
                              below 1e-6); 0 (default): 3e-6 for VIE_FP32, 1e-3
                              for VIE_FP16, 8e-3 for VIE_BF16                     */
    int32_t timing;        /* 1: record CUDA events around the main kernels and
                              report their device times in vie_result.k_* (adds
                              no work, only events on the solve stream)          */
    int32_t precond_block_max;  /* 0 (default): one block per material domain,
                              the preconditioner of Eq. (6).  > 0: sub-block
                              variant (not in the paper): a domain with more
                              unknowns than this is cut into spatially compact
                              sub-blocks of at most this many (recursive
                              coordinate bisection of the unknowns' positions),
                              each inverted and applied as its own diagonal
                              block; inversion work drops by about the square of
                              the number of pieces, GMRES may need more
                              iterations                                         */
    int32_t precond_pivot; /* outer pivot width of the block inversion: 512 or
                              1024 sets it; 0 (default): 512, or the width
                              vie_tune chose for the mesh                        */
    int32_t autotune;      /* 1: the first solve of each incidence class (normal,
                              oblique) on a mesh first runs vie_tune on its own
                              request (vie_solve_batch: before its slots start),
                              and the mesh's later solves use the choices; 0
                              (default): the built-in schedule                   */
} vie_options;

typedef struct {
    double  lambda_nm;                  /* vacuum wavelength                       */
    double  theta;                      /* polar angle of incidence [rad]          */
    double  phi;                        /* azimuth of the plane of incidence [rad] */
    double  eps[2 * VIE_MAX_DOMAINS];   /* per-domain relative permittivity (re,im)*/
    double *coeffs_out;                 /* optional [N][2 pol] complex (re,im): the
                                           solved unknowns in canonical order; host
                                           pointer, or device if coeffs_on_device */
    int32_t coeffs_on_device;
    int32_t density_on_device;          /* density_out is a device pointer          */
    double *density_out;                /* optional [2 pol][n_tets]: the absorbed
                                           fraction of Eq. (7) contributed by each
                                           tetrahedron, k0 |Im eps_r| int_t |E|^2 dV
                                           / (|E0|^2 a b cos theta) (the absorption
                                           profile of Fig. 5); the sum over the
                                           tetrahedra of a domain is absorbed[p][d]  */
} vie_request;

typedef struct {
    int32_t status;                      /* vie_status of the solve                 */
    int32_t n_unknowns;
    int32_t iterations[2];               /* GMRES iterations, TE and TM             */
    int32_t refinements;                 /* outer FP64 refinement sweeps            */
    double  rel_residual[2];             /* final FP64 ||b - Z x|| / ||b||          */
    double  absorbed[2][VIE_MAX_DOMAINS];/* fraction of incident power per domain   */
    double  reflectance[2];
    double  transmittance[2];
    double  t_fill_ms, t_factor_ms, t_solve_ms, t_post_ms;   /* host wall time per phase */
    /* device times from CUDA events on the solve stream (options.timing = 1):
       k_far_tt_ms   the far tetrahedron-pair fill kernel (one launch)
       k_fill_ms     the whole fill (all fill kernels)
       k_factor_ms   the whole block inversion
       k_matvec_ms   total of the Z matvec launches in GMRES, k_matvec_n launches */
    double  k_far_tt_ms, k_fill_ms, k_factor_ms, k_matvec_ms;
    int32_t k_matvec_n;
    int32_t n_near_pairs;                /* near tetrahedron pairs of the mesh       */
    int64_t far_pair_evals;              /* Green's-function evaluations of the
                                            tetrahedron-pair kernel (16 per pair)   */
    int64_t h2d_bytes, d2h_bytes;        /* host<->device bytes this solve copied    */
    /* tensor-core products of the block inversion (options.timing = 1): total
       device time of the k_tc_n timed launches (trailing/row-panel products)
       and their algorithmic bytes (read and write of the updated block plus
       one read of the two operand panels) */
    double  k_tc_ms, k_tc_bytes;
    int32_t k_tc_n;
    int32_t n_launches;                  /* CUDA kernels this call launched          */
    /* solve server only (0 elsewhere): time from vie_server_submit to the start
       of the solve, and to its end */
    double  t_queue_ms, t_latency_ms;
    /* applications of the preconditioner of Eq. (6) in GMRES (options.timing = 1):
       total device time of the k_precond_n applications and their algorithmic
       bytes (one read of every block inverse plus the vectors) */
    double  k_precond_ms, k_precond_bytes;
    int32_t k_precond_n, reserved3;
    double  k_tc_flops;                  /* algorithmic flops of the k_tc_n launches */
    /* GMRES orthogonalisation (options.timing = 1): total device time of the
       classical Gram-Schmidt passes (both projections, both updates and the
       norm of the new vector) over all iterations */
    double  k_ortho_ms;
} vie_result;

/* Fill *opt with defaults (FP32 with refinement, preconditioner on, tol 1e-6,
   restart 100, max_iter 1000, inner_tol 0 = per precision). */
void vie_default_options(vie_options *opt);

/* Create a context on CUDA device `device`.  opt may be NULL (defaults).
   *out receives the context; returns VIE_OK or an error code. */
int vie_create(vie_ctx **out, int device, const vie_options *opt);

/* Replace the solver options of an existing context. */
int vie_set_options(vie_ctx *ctx, const vie_options *opt);

/* Mesh of one unit cell (Fig. 1): verts [n_verts][3] (nm), tets [n_tets][4]
   positively oriented, tet_domain [n_tets] in 0..n_domains-1; period a x b;
   active_domain = the domain whose absorption Eq. (7) reports.  The lateral
   walls x=0/a and y=0/b must carry matching triangulations.  Builds the SWG
   topology (Sec. 2.1) and the near-pair lists; keeps them on the device. */
int vie_set_mesh(vie_ctx *ctx, const double *verts, int32_t n_verts,
                 const int32_t *tets, int32_t n_tets,
                 const int32_t *tet_domain, int32_t n_domains,
                 double period_a, double period_b, int32_t active_domain);

/* Number of SWG unknowns of the current mesh (0 before vie_set_mesh). */
int32_t vie_num_unknowns(const vie_ctx *ctx);

/* One solve at one incidence for TE and TM together: fill Eq. (2) with the
   Ewald-summed g_p (Eq. (3)-(4)), factor the domain blocks (Eq. (6)), run
   GMRES, compute Eq. (7) absorption per domain plus R and T.
   stream: a cudaStream_t (may be NULL for the legacy default stream); the call
   returns after the work on it has finished.  The block inversion and the
   preconditioner applications also use two non-blocking streams that the
   context owns (look-ahead, and the smaller domain blocks beside the
   largest); their work is ordered after, and joined back into, `stream` by
   events, so nothing of the solve is left running when the call returns. */
int vie_solve(vie_ctx *ctx, const vie_request *req, vie_result *res, void *stream);

/* A batch of independent solves on the current mesh (a wavelength x angle
   sweep): reqs[n] in, res[n] out (caller-owned; res[i] is what vie_solve
   would return for reqs[i], status included).  Up to max_slots solves run at
   once, each in its own solve slot: a host thread, a CUDA stream and its own
   device copy of Z, the block inverses of Eq. (6) and the Krylov state, all
   reading the one device copy of the mesh.  One request's fill overlaps the
   block inversion and GMRES of others.  Slots are opened while their device
   footprint (estimated from reqs[0]) fits in free HBM less 5% and 1 GB; the
   context keeps them, with their buffers, for later batches until
   vie_destroy.  *slots_used (may be NULL)
   receives the number of slots that ran.  The caller's stream is synchronised
   before the first solve; the call returns when all solves have finished.
   Returns VIE_OK, the first negative status of a request, or else the first
   positive one. */
int vie_solve_batch(vie_ctx *ctx, const vie_request *reqs, vie_result *res, int32_t n,
                    int32_t max_slots, int32_t *slots_used, void *stream);

/* Autotuner (not in the paper; the schedule of this implementation): times
   candidate schedules of the two hot parts on the context's mesh and on `req`
   with CUDA events on `stream`, and keeps the fastest for the mesh (every later
   vie_solve / vie_solve_batch of this context uses them; vie_set_mesh resets
   them).  Tuned, per incidence class of req (normal: theta = 0, or oblique):
   - the fill: the Ewald split multiplier E / sqrt(pi / ab) of the FP32 tables
     (normal 1.25, 1.5, 1.75; oblique 1.0, 1.25, 1.5): it moves work between
     the lattice images and the Floquet orders, the value of the matrix does not
     change (the series is split, not truncated differently); each candidate
     is timed over a whole fill (best of two); VIE_FP64 keeps its own split;
   - the GMRES products: 1, 2 or 4 row ranges per resident CTA (mean of five
     products of the matrix the products read);
   - once per mesh, where a domain block has more than 1024 unknowns: the outer
     pivot width of the block inversion of Eq. (6), 512 or 1024 (half the
     passes over the block against a longer chain of pivot-block inverses),
     each over a whole inversion (best of two).
   It fills Z (the request's matrix; the next solve fills it again) and
   allocates two vectors.  report (optional, caller-owned) receives every
   candidate's time and the choices.  Errors as vie_solve (a candidate whose
   tables do not fit is skipped and reported with fill_ms = -1). */
typedef struct {
    int32_t incidence_class;   /* 0: normal incidence, 1: oblique                   */
    int32_t n_split;           /* candidates of the split timed (0 for VIE_FP64)    */
    double  split[4];          /* multiplier of sqrt(pi / ab)                        */
    double  fill_ms[4];        /* device time of the whole fill with it (-1: skipped)*/
    double  split_chosen;
    int32_t n_mv;
    int32_t mv_grid[4];        /* row ranges per resident CTA of the GMRES products  */
    double  mv_ms[4];          /* device time of one product with it                 */
    int32_t mv_chosen;
    int32_t n_pivot;           /* 0: pivot width not timed (already tuned for the
                                  mesh, no block wider than 1024, or no
                                  preconditioner)                                   */
    int32_t pivot[2];          /* outer pivot width of the block inversion           */
    double  factor_ms[2];      /* device time of the whole block inversion with it   */
    int32_t pivot_chosen;      /* the width the mesh's solves use                    */
    double  tune_ms;           /* host wall time of the tuning                       */
} vie_tune_report;
int vie_tune(vie_ctx *ctx, const vie_request *req, vie_tune_report *report, void *stream);

/* Parity entry points: the FP64 impedance matrix Z [N][N] (row-major, complex)
   and right-hand side b [N][2] of Eq. (2) in canonical unknown order, copied
   to host buffers owned by the caller.  They run the same fill kernels as
   vie_solve in FP64. */
int vie_fill_matrix(vie_ctx *ctx, const vie_request *req, double *Z_host, double *b_host, void *stream);

/* Parity entry point: the matrix in the precision of the current options,
   widened to double, canonical order: the FP32 Z (VIE_FP32), or the 16-bit
   copy the GMRES products read with its scale undone (VIE_FP16, VIE_BF16). */
int vie_fill_matrix_prec(vie_ctx *ctx, const vie_request *req, double *Z_host, void *stream);

/* Parity entry point for the preconditioner of Eq. (5)-(6): fills Z for the
   request in the precision of the current options, inverts every domain block
   as vie_solve does, and returns block `block` (0-based, in increasing domain
   order over the non-empty domains, unknowns grouped by the Eq. (5) rule; with
   options.precond_block_max > 0 the sub-blocks of each domain in turn):
   *n_out its size n; unknowns [n] (may be NULL) the canonical index of its
   row/column i; Zdd [n][n] complex (may be NULL) the block A_dd as stored
   (FP32 or FP64 entries widened); Minv [n][n] complex (may be NULL) the
   computed inverse (FP32, before its FP16 copy).  With all three NULL only
   *n_out is set (no fill).  VIE_EINVAL for a block index out of range. */
int vie_domain_block(vie_ctx *ctx, const vie_request *req, int32_t block, int32_t *n_out, int32_t *unknowns,
                     double *Zdd, double *Minv, void *stream);

/* Check of the failure path of the device's bounded waits (the paper has no
   counterpart): one thread waits, with the bounded mbarrier wait the
   tensor-core block inversion uses, on a barrier that gets its arrival
   (arrive = 1) or never does (arrive = 0), for at most `polls` polls
   (1..1000000).  Returns VIE_OK when the wait completed, VIE_DEVICE_TIMEOUT
   when it ran out (the kernel gave up and returned; the device stays usable),
   VIE_EINVAL or VIE_ECUDA. */
int vie_check_device_wait(int device, int32_t arrive, int32_t polls);

/* Measured peak of the FP32 (precision VIE_FP32) or FP64 (VIE_FP64) fused
   multiply-add pipes of `device`, in TFLOP/s, from a kernel of independent FMA
   chains on every SM (the best of three launches of at least 100 ms each):
   the denominator of the roofline of the CUDA-core fill kernels.  The paper
   has no counterpart; a measurement entry point.  Allocates nothing; uses a
   stream and two events of its own.  Returns VIE_OK, VIE_EINVAL or VIE_ECUDA. */
int vie_fma_peak(int device, int32_t precision, double *tflops);

/* Complex erfcx(u) = exp(u^2) erfc(u) = w(j u) on the device for n host
   arguments (Re u >= 0), in FP64 (precision VIE_FP64) or FP32 (VIE_FP32).
   Used to check the Faddeeva evaluation of the Ewald series. */
int vie_erfcx(vie_ctx *ctx, const double *u, double *out, int32_t n, int32_t precision);

/* The Ewald-summed periodic Green's function g_p(d), Eq. (3), on the device
   for n in-cell difference vectors d [n][3] (|dx| < a, |dy| < b, d != 0) at
   the request's wavelength and incidence; out [n] complex.  VIE_FP32 takes the
   evaluation form the fill kernels take for that incidence (the short normal
   or oblique form where it applies, else the general tabulated form), so it
   checks the fill's own arithmetic. */
int vie_green(vie_ctx *ctx, const vie_request *req, const double *d, double *out,
              int32_t n, int32_t precision);

/* Allocation-free g_p(d): the same Ewald series as vie_green (in FP32 the
   general tabulated form, where vie_green takes the fill's short form: the two
   agree to the FP32 accuracy of the tables, 2e-6 max|g| each), for callers
   that cannot allocate device memory while they run (a host framework that
   owns all of HBM through its own pool and forbids cudaMalloc/cudaFree after
   start-up, or code that must not let an allocation synchronise the device).
   The paper has no counterpart; this is a deployment entry point.
   Arguments: incidence (lambda_nm, theta, phi) as in vie_request; lattice
   periods period_a, period_b (nm); z_extent >= the largest |dz| that will be
   evaluated (the FP32 tables cover |dz| in [0, z_extent]); d_dev [n][3] and
   out_dev [n] complex (re,im) are DEVICE buffers owned by the caller, with the
   same in-cell restriction as vie_green; precision VIE_FP64 or VIE_FP32;
   stream a cudaStream_t (NULL: legacy default stream).  Needs no context.
   Scratch: the Ewald parameter block and the FP32 interpolation tables live
   in a file-scope device array of about 0.85 MB that every GPU loading this
   library keeps until the process exits; requests needing more than 96
   distinct Floquet decay constants are rejected with VIE_EINVAL.  The tables
   are rebuilt completely by each call, so nothing has to start at zero.  All
   calls share that array: calls whose work overlaps on the GPU race.
   The first call on a device (the current device) does a one-time set-up,
   under a lock shared by all host threads: the library's constant tables (the
   same once-per-device upload vie_create does; a device that already has them
   is not written again) and the device address of the array.  Make that first
   call before any stream capture.  Each call copies the Ewald parameter block
   (~49 KB) from host memory of the calling thread to the array on `stream`
   (a pageable copy: the call can wait for it to be staged); the table build
   and the evaluation are then enqueued on `stream`, and out_dev is valid once
   the stream has completed them.  Calls no cudaMalloc, cudaFree or allocating
   library routine.  Returns VIE_OK, VIE_EINVAL, VIE_RAYLEIGH_ANOMALY or
   VIE_ECUDA. */
int vie_green_noalloc(double lambda_nm, double theta, double phi, double period_a, double period_b,
                      double z_extent, const double *d_dev, double *out_dev, int32_t n,
                      int32_t precision, void *stream);

/* ------------------------------------------------------------------------
   Solve server: continuous batching of independent solves, each with its own
   mesh (a stream of (geometry, lambda, theta) requests of different sizes).
   The paper solves one configuration at a time; this is a deployment layer
   over vie_set_mesh + vie_solve.

   A server owns n_slots solve slots on one device.  Each slot is a host
   thread with its own context (mesh, Z, block inverses of Eq. (6), Krylov
   state, all device resident) and its own CUDA stream, so the solves of
   different slots overlap on the GPU.  A queued request is admitted to a free
   slot as soon as its device footprint fits in the HBM budget next to what
   the other slots hold: requests are taken in arrival order, and a later
   request that fits may pass one that does not (at most 8 times per waiting
   request, then the queue waits for it).  All server functions are thread
   safe. */

typedef struct vie_server vie_server;

typedef struct {                 /* one unit-cell mesh, as in vie_set_mesh    */
    const double  *verts;        /* [n_verts][3] nm                           */
    int32_t        n_verts;
    const int32_t *tets;         /* [n_tets][4]                               */
    int32_t        n_tets;
    const int32_t *tet_domain;   /* [n_tets]                                  */
    int32_t        n_domains;
    int32_t        active_domain;
    double         period_a, period_b;
} vie_mesh;

typedef struct {
    int64_t submitted, completed, rejected;   /* requests                        */
    int64_t queued, running, max_running;     /* now, and the most at once       */
    int64_t budget_bytes;                     /* HBM budget of the slots          */
    int64_t reserved_bytes, peak_reserved_bytes;
    int64_t cancelled;                        /* requests that ended VIE_CANCELLED */
} vie_server_stats;

/* Start a server on `device` with n_slots slots (1..64) and solver options
   opt (NULL: defaults).  hbm_budget_bytes bounds the device memory the slots
   may hold together; 0 means the free memory at creation less 5% and 1 GB. */
int vie_server_create(vie_server **out, int device, const vie_options *opt, int32_t n_slots,
                      int64_t hbm_budget_bytes);

/* Queue one request: the mesh and the request are copied (except
   req->coeffs_out, which must stay valid until the request has finished).
   *ticket receives its id; *footprint_bytes (may be NULL) the device bytes
   its slot will hold (an upper bound computed from the mesh: Z, block
   inverses, Krylov basis, near-pair masks).  Returns VIE_OK, VIE_EINVAL, or
   VIE_ENOMEM when the footprint exceeds the whole budget (not queued). */
int vie_server_submit(vie_server *s, const vie_mesh *mesh, const vie_request *req, uint64_t *ticket,
                      int64_t *footprint_bytes);

/* Wait up to wait_ms (0: do not wait, negative: until done) for a request.
   Returns VIE_OK with *res filled (res->status is the solve's status, the
   ticket is then forgotten), VIE_PENDING if it has not finished, VIE_EINVAL
   for an unknown ticket. */
int vie_server_poll(vie_server *s, uint64_t ticket, vie_result *res, int32_t wait_ms);

/* Cancel a request: a queued request is dropped, a running one stops at its
   next GMRES iteration (or before its next phase); either way the ticket then
   polls as finished with res->status = VIE_CANCELLED.  A request that had
   already finished keeps its result.  Returns VIE_OK, or VIE_EINVAL for an
   unknown ticket. */
int vie_server_cancel(vie_server *s, uint64_t ticket);

/* Counters of the server (a snapshot). */
int vie_server_get_stats(vie_server *s, vie_server_stats *out);

/* Finish the solves in progress, drop queued requests, free everything. */
void vie_server_destroy(vie_server *s);

/* Human-readable name of a status code; never NULL. */
const char *vie_status_str(int status);

/* Description of the last error on ctx (empty string if none); never NULL. */
const char *vie_last_error(const vie_ctx *ctx);

/* Free all device and host memory of the context. */
void vie_destroy(vie_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* VIE_H */
