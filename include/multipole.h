/*
 * multipole.h -- C ABI of the GB300 multipole Poisson solver.
 *
 * Solves nabla^2 Phi = S, S = 4 pi G rho, for an isolated source on a spherical
 * (r, theta, phi) mesh with the multipole method of GenASiS II (Cardall,
 * Budiardja, Murphy & Endeve), Sec. 2.2:
 *   (a) angular moments of each radial shell, Eq. (AngularMomentsDiscrete),
 *       with cell-averaged real kernels A^c_lm = P~_l^m cos(m phi),
 *       A^s_lm = P~_l^m sin(m phi), Eqs. (AngularKernel_c), (AngularKernel_s);
 *   (b) weighting by the shell integrals of r^l and r^-(l+1),
 *       Eqs. (RadialRegular), (RadialIrregular);
 *   (c) outward (regular) and inward (irregular) radial recurrences on the
 *       n_r + 1 shell edges;
 *   (d) the potential at every cell, Eq. (Solution), from the edge moments
 *       interpolated to the cell centre.
 * All compute runs in CUDA kernels on the device; there is no CPU fallback.
 *
 * Layouts (C row-major, float64 unless stated):
 *   rho, phi       [n_r][n_theta][n_phi]
 *   moments        [n_r][K_L]         K_L = (L+1)^2 real moments per shell
 *   edge moments   [n_r + 1][K_L]
 *   moment index   q(l,m,a) = l*l + p(m,a), p(0,c) = 0, p(m,c) = 2m-1,
 *                  p(m,s) = 2m (m >= 1); the (m = 0, sine) kernel vanishes
 *                  identically and is not carried.
 *
 * Conventions the paper leaves open (each is documented with the library):
 *   - cell averages of the angular kernels are solid-angle means and those of
 *     the radial kernels volume means;
 *   - "linear interpolation to the cell center" uses the coordinate midpoint;
 *   - radial kernels are scaled by r_ref = sqrt(r_min+ * r_max) (r_min+ the
 *     smallest positive edge): R^R -> (r/r_ref)^l, R^I -> r_ref^l / r^(l+1); the
 *     exported edge moments M^R, M^I carry that scaling, Phi does not depend
 *     on it;
 *   - a shell touching r = 0 replaces, for l >= 2, its divergent own-shell
 *     term by 6 r_1^2 / (5 (l + 3)) times the shell's moment (the exact volume
 *     mean for a moment uniform inside the ball); M^I at edge 0 then excludes
 *     that shell's own term.
 *
 * Threading and ordering: a mesh is bound to one CUDA stream; every call that
 * touches the device is enqueued on it and returns without waiting unless its
 * comment says otherwise.  Calls on one mesh must not run concurrently from
 * several host threads.  Device-side errors (non-finite density, a wait that
 * ran out of time) are recorded on the device and reported by the next
 * mp_mesh_synchronize() or mp_solve_host().
 *
 * Errors: every function returns an mp_status.  Argument errors are detected on
 * the host before anything is enqueued and leave the mesh unchanged.
 * mp_last_error_detail() gives a one-line explanation of the last error raised
 * on the calling host thread.
 */
#ifndef GB300_MULTIPOLE_H
#define GB300_MULTIPOLE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MP_API __attribute__((visibility("default")))
#else
#define MP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mp_mesh mp_mesh;   /* opaque, library-owned */
typedef struct mp_batch mp_batch; /* opaque, library-owned */

typedef enum {
    MP_OK = 0,
    MP_ERR_INVALID_ARG = 1, /* a pointer, size or edge array is unusable            */
    MP_ERR_RANGE = 2,       /* r^l or r^-(l+1) would leave the float64 range         */
    MP_ERR_CUDA = 3,        /* a CUDA runtime call failed                           */
    MP_ERR_OOM = 4,         /* device or host allocation failed                     */
    MP_ERR_NOT_READY = 5,   /* no density bound yet                                 */
    MP_ERR_NONFINITE = 6,   /* the density held a NaN or an infinity                */
    MP_ERR_TIMEOUT = 7,     /* a device-side wait gave up (pipeline stalled)         */
    MP_ERR_UNSUPPORTED = 8  /* valid request this build cannot serve (see detail)   */
} mp_status;

typedef enum {
    MP_PREC_FP64 = 0,   /* every step in float64 on CUDA cores                       */
    MP_PREC_BF16X3 = 1, /* angular contractions as split-bf16 tensor-core GEMMs,     */
                        /* density deviations in 2 bf16 terms, tables in 3           */
    MP_PREC_BF16X6 = 2  /* as BF16X3 with 3 bf16 terms on both operands              */
} mp_precision;

/* Sizes and the effective configuration of a mesh (mp_mesh_get_info). */
typedef struct {
    int n_r, n_theta, n_phi, l_max;
    int n_moments;           /* K_L = (l_max + 1)^2                                  */
    int precision;           /* requested mp_precision                               */
    int effective_precision; /* what solve runs: split meshes with odd n_phi run FP64 */
    double r_ref;            /* reference radius of the radial kernel scaling        */
    double G;                /* gravitational constant, S = 4 pi G rho               */
    size_t device_bytes;     /* device memory the mesh holds (tables + workspace)    */
    int tuned_candidates;    /* configurations the last mp_autotune timed (0: none,  */
                             /* or the choice came from the cache file)              */
    int theta_tensor_cores;  /* 1: the split path runs the theta stages of the       */
                             /* orders m >= 1 on the tensor cores (tcgen05)          */
} mp_mesh_info;

/*
 * Create a mesh and build its tables on the device in float64 (Sec. 2.2: the
 * cell-averaged angular kernels and the analytically averaged radial kernels
 * are computed once and stored).
 *   r_edges      host, n_r + 1 values, strictly increasing, r_edges[0] >= 0.
 *   theta_edges  host, n_theta + 1 values, strictly increasing within [0, pi].
 *   phi_edges    host, n_phi + 1 values, strictly increasing, span <= 2 pi.
 *                (The source is taken to vanish outside the meshed angles.)
 *   l_max        0 <= l_max <= 128; the split precisions need 2 l_max + 1 <= 256.
 *   G            gravitational constant (> 0).
 *   prec         mp_precision.
 *   cuda_stream  cudaStream_t to enqueue on (NULL = legacy default stream).
 *   out          receives the mesh; unchanged on error.
 * The edge arrays are copied.  Blocks until the tables are built.
 * Errors: MP_ERR_INVALID_ARG, MP_ERR_RANGE, MP_ERR_OOM, MP_ERR_CUDA.
 */
MP_API mp_status mp_mesh_create(const double *r_edges, int n_r, const double *theta_edges, int n_theta,
                         const double *phi_edges, int n_phi, int l_max, double G, mp_precision prec,
                         void *cuda_stream, mp_mesh **out);

/*
 * Radial-shell domain decomposition (Sec. 2.1: the mesh is divided among processes
 * into radial shells that each cover the full solid angle; Sec. 2.2: the moment sums
 * are then combined across processes).  A slab holds shells [i0, i1) of a mesh whose
 * n_r + 1 radial edges are r_edges; its radial kernels use the whole mesh's reference
 * radius, so that the radial sums of different slabs add.  The radial recurrences of
 * the whole mesh differ from a slab's own only by two constants per moment: the sum of
 * W^R A over the slabs below it (added to every M^R edge) and the sum of W^I A over the
 * slabs above it (added to every M^I edge).  A solve over P slabs is therefore
 *   1. on every slab: mp_slab_moments -> its totals T[2][K_L] (device):
 *      T[0][q] = sum over its shells of W^R_l A_q, T[1][q] = sum of W^I_l A_q;
 *   2. one exclusive prefix over the slabs in radial order (2 K_L doubles each):
 *      outer[0][q] = sum of T[0][q] over the slabs below, outer[1][q] = sum of T[1][q]
 *      over the slabs above (paper_2602_02507_gb300.sharding does it with
 *      torch.distributed, one slab per rank);
 *   3. on every slab: mp_slab_potential(outer) -> its edge moments, coefficients
 *      and Phi, equal to the whole mesh's on its shells up to rounding.
 * Arguments as mp_mesh_create, plus 0 <= i0 < i1 <= n_r.  The slab's density and
 * potential cover only its shells ([i1 - i0][n_theta][n_phi]); mp_solve on a slab
 * solves it alone (no other slabs).  Errors as mp_mesh_create.
 */
MP_API mp_status mp_mesh_create_slab(const double *r_edges, int n_r, int i0, int i1, const double *theta_edges,
                                     int n_theta, const double *phi_edges, int n_phi, int l_max, double G,
                                     mp_precision prec, void *cuda_stream, mp_mesh **out);

/* Step 1 above: angular moments of the bound density and this slab's radial totals
 * (totals_dev: device [2][K_L], written on the mesh's stream).  Any mesh may call it.
 * Errors: MP_ERR_INVALID_ARG, MP_ERR_NOT_READY (no density bound). */
MP_API mp_status mp_slab_moments(mp_mesh *mesh, double *totals_dev);

/* Step 3 above: outer_dev (device [2][K_L]) holds the sums of the other slabs; writes
 * the potential into the bound output and keeps the edge moments for mp_get_moments.
 * Errors: MP_ERR_INVALID_ARG, MP_ERR_NOT_READY (mp_slab_moments has not run since the
 * last call). */
MP_API mp_status mp_slab_potential(mp_mesh *mesh, const double *outer_dev);

/* Release the mesh and every device buffer it owns (waits for its stream). */
MP_API mp_status mp_mesh_destroy(mp_mesh *mesh);

/* Rebind the mesh to another stream (waits for work on the old one first). */
MP_API mp_status mp_mesh_set_stream(mp_mesh *mesh, void *cuda_stream);

/* Sizes and configuration; host only, never touches the device. */
MP_API mp_status mp_mesh_get_info(const mp_mesh *mesh, mp_mesh_info *info);

/*
 * Bind the density: device pointer to n_r * n_theta * n_phi float64 values in
 * the rho layout.  Nothing is copied: the buffer is read by each later
 * mp_solve() and must stay valid until then.  Caller owns it.
 */
MP_API mp_status mp_set_density(mp_mesh *mesh, const double *rho_dev);

/*
 * Bind the output: device pointer to n_r * n_theta * n_phi float64 values that
 * later mp_solve() calls write Phi into (caller owns it).  NULL makes the mesh
 * write into a buffer of its own, allocated on first use.
 */
MP_API mp_status mp_set_phi_output(mp_mesh *mesh, double *phi_dev);

/*
 * Run steps (a)-(d) on the mesh's stream: reads the bound density, writes Phi
 * and keeps the moments of this solve for mp_get_moments().  The kernel chain
 * is captured once as a CUDA graph (on a private stream, at the first solve
 * and again after the bound buffers change or mp_autotune) and replayed by one
 * graph launch per solve; with profiling enabled the kernels are launched one
 * by one instead, with events between them.
 * Errors: MP_ERR_NOT_READY (no density bound), MP_ERR_OOM, MP_ERR_CUDA;
 * device-side errors surface at mp_mesh_synchronize().
 */
MP_API mp_status mp_solve(mp_mesh *mesh);

/*
 * Copy the last Phi into phi_dev (device pointer, rho layout).  A no-op when
 * phi_dev is the bound output buffer.  Stream-ordered.
 */
MP_API mp_status mp_get_phi(mp_mesh *mesh, double *phi_dev);

/*
 * Copy the moments of the last solve (device pointers; any may be NULL):
 *   ang_dev [n_r][K_L]      angular moments of step (a), Eq. (AngularMomentsDiscrete)
 *   mr_dev  [n_r + 1][K_L]  regular (outward) edge moments of step (c)
 *   mi_dev  [n_r + 1][K_L]  irregular (inward) edge moments of step (c)
 * Stream-ordered.
 */
MP_API mp_status mp_get_moments(mp_mesh *mesh, double *ang_dev, double *mr_dev, double *mi_dev);

/*
 * End-to-end solve from host memory: copies rho_host to the device, solves,
 * copies Phi back into phi_host and waits for completion (both host arrays in
 * the rho layout; pinned memory gives the fastest copies).  Returns any
 * device-side error of the solve.
 */
MP_API mp_status mp_solve_host(mp_mesh *mesh, const double *rho_host, double *phi_host);

/*
 * The same round trip without waiting: the upload, the solve and the download
 * are enqueued and the call returns.  The mesh keeps two device staging pairs
 * and uses them in turn, with the uploads and downloads on streams of its own,
 * so that the download of one call overlaps the upload of the next.  rho_host
 * must stay unchanged and phi_host unread until mp_mesh_synchronize() (which
 * also reports device-side errors); both should be pinned for the copies to run
 * asynchronously.  mp_get_phi() then returns the last call's Phi.
 */
MP_API mp_status mp_solve_host_async(mp_mesh *mesh, const double *rho_host, double *phi_host);

/* Wait for the mesh's stream and return (then clear) any device-side error. */
MP_API mp_status mp_mesh_synchronize(mp_mesh *mesh);

/*
 * Engine of the theta factors of both angular contractions on the split path
 * (Eq. (AngularMomentsDiscrete) and Eq. (Solution), the sums over polar cells and
 * over degrees): 1 runs the orders m >= 1 as split-bf16 tcgen05 GEMMs, one per order
 * (the m = 0 column stays on CUDA cores in compensated float32 / double-float);
 * 2 runs every order on CUDA cores in float32; 0 restores the mesh's default (the
 * tensor cores where the CUDA-core kernels cannot keep their tables in shared memory).
 * mp_autotune also times both.  Both give results within the split-path tolerance;
 * they differ in rounding.  Waits for the mesh's stream; later solves re-capture
 * their graph.  Errors: MP_ERR_INVALID_ARG (engine outside 0..2), MP_ERR_UNSUPPORTED
 * (1 on a float64 mesh, or l_max = 0).
 */
MP_API mp_status mp_set_theta_engine(mp_mesh *mesh, int engine);

/*
 * Failure detection: every wait inside the split-precision kernels (on a copy,
 * an MMA or another warp role of the same block) is bounded.  When one runs past
 * the budget the block records MP_ERR_TIMEOUT in the mesh's device error word,
 * lets every copy and MMA it issued finish (with the full default budget), frees
 * its tensor memory and exits; mp_mesh_synchronize() then returns
 * MP_ERR_TIMEOUT and the mesh stays usable.  This sets that budget in SM clock
 * cycles for later solves of the mesh; cycles <= 0 restores the default of
 * 2e9 cycles (about a second at the boost clock).  A tiny budget makes the
 * waits run out on purpose, which is how the abort path is tested.  The paper
 * has no counterpart.  Waits for the mesh's stream first; blocks until set.
 */
MP_API mp_status mp_set_wait_budget(mp_mesh *mesh, long long cycles);

/*
 * Per-kernel timing on the mesh's stream (CUDA events around each launch).
 * mp_profile_enable(mesh, 1) starts recording (and resets totals);
 * mp_profile_read() waits for the stream, then fills up to cap entries with
 * kernel names (static strings), launch counts and total milliseconds and
 * returns the number of distinct kernels in *n_out.
 */
MP_API mp_status mp_profile_enable(mp_mesh *mesh, int enable);
MP_API mp_status mp_profile_read(mp_mesh *mesh, const char **names, int *launches, double *total_ms, int cap,
                          int *n_out);

/*
 * Batched solves: many meshes (uneven sizes and l_max, each with its density
 * and output bound) solved together.  The first mesh's stream is used.  The
 * whole batch is replayed as one captured CUDA graph after the first solve.
 *   meshes  host array of count mesh pointers (borrowed: they must outlive
 *           the batch and keep their bindings).
 */
MP_API mp_status mp_batch_create(mp_mesh *const *meshes, int count, mp_batch **out);
MP_API mp_status mp_batch_solve(mp_batch *batch);
MP_API mp_status mp_batch_destroy(mp_batch *batch);

/*
 * Pick launch parameters for the mesh by timing candidates on the device
 * (needs a bound density).  Swept: the projection's density ring depth, its
 * table residency and its number of TMEM accumulators; the phi synthesis's
 * stage configuration (A-operand stages, table residency or ring depth, and
 * the count and width of its output staging boxes); the threads per moment
 * column of the radial recurrences; the engine of the theta stages (tensor
 * cores or CUDA cores, see mp_set_theta_engine) and the shells per unit of
 * the tensor-core theta synthesis.  The choice is cached in cache_path (a
 * text file, may be NULL; one line per mesh key, ending in the format tag
 * "s2", lines of other formats ignored) keyed by (n_r, n_theta, n_phi, l_max,
 * precision) and reused by later meshes of the same key.  A cached line that
 * does not fit the mesh's plan is skipped, and the candidates are timed anew.
 */
MP_API mp_status mp_autotune(mp_mesh *mesh, const char *cache_path);

/*
 * Gravitational source terms of the fluid balance equations (Sec. 3,
 * Eq. (BalancedVariablesGravitational)) from a potential on this mesh:
 *   grad[a] = d(Phi)/dx^a, x = (r, theta, phi)   (coordinate derivatives)
 *   S[a]    = -rho grad[a]                        (momentum source, covariant)
 *   E       = -rho (v^r grad[0] + v^theta grad[1] + v^phi grad[2])  (energy source)
 * Each derivative is the centred difference over the two nearest cells along
 * the coordinate (the rule Sec. 3 states with the sources), with cell centres
 * at coordinate midpoints: (Phi[hi] - Phi[lo]) / (x_c[hi] - x_c[lo]).  phi
 * wraps around when the azimuthal edges span 2 pi; at the ends of r, theta (and
 * of a shorter azimuthal range) the two nearest cells are the cell and its one
 * neighbour.  One cell along a coordinate, or two azimuthal cells on a full
 * circle, give a zero derivative.
 *   phi_dev  [n_r][n_theta][n_phi] float64, device; NULL: the last solve's Phi
 *   rho_dev  same layout; NULL: the bound density
 *   v_dev    [3][n_r][n_theta][n_phi] (v^r, v^theta, v^phi), or NULL
 *   grad_dev, S_dev [3][n_r][n_theta][n_phi]; E_dev [n_r][n_theta][n_phi]:
 *            outputs, each may be NULL (not all; E_dev needs v_dev); they must
 *            not overlap the inputs
 * All buffers are caller-owned device memory; nothing is allocated.  Float64
 * arithmetic whatever the mesh precision.  Enqueued on the mesh's stream;
 * argument errors return at once (MP_ERR_INVALID_ARG, or MP_ERR_NOT_READY when
 * phi_dev is NULL before any solve or rho_dev is NULL with no bound density).
 */
MP_API mp_status mp_gravity_sources(mp_mesh *mesh, const double *phi_dev, const double *rho_dev, const double *v_dev,
                                    double *grad_dev, double *S_dev, double *E_dev);

/*
 * Coarsening-block averaging (Sec. 2.1, where angular cell widths fall below the
 * minimum radial width cells are grouped into angular blocks at each radius;
 * Sec. 2.3, each cell of a block takes the block's volume-weighted mean
 * sum V_j K_j / sum V_j, which conserves the block's integral).  Blocks, a reading
 * of the paper's figures: with Delta r_min the smallest radial width and widths at
 * the cell-centre radius r_c, polar blocks are runs of p cells, p the smallest
 * power of two dividing n_theta with p r_c min(dtheta) >= Delta r_min (else the
 * whole polar range); within a polar block, azimuthal blocks are runs of q cells,
 * q the smallest power of two dividing n_phi with q r_c sin(theta_c) min(dphi) >=
 * Delta r_min for the block's cell nearest the axis (else the whole ring).
 *   fields_dev  n_fields device arrays of [n_r][n_theta][n_phi] float64, the f-th
 *               at fields_dev + f * field_stride; averaged in place (cells outside
 *               every block are not touched)
 * Float64; nothing is allocated; enqueued on the mesh's stream.
 */
MP_API mp_status mp_coarsen(mp_mesh *mesh, double *fields_dev, int n_fields, long long field_stride);

/*
 * The block sizes of mp_coarsen (host arrays, caller-owned; either may be NULL):
 * c_theta [n_r] polar block size per shell, c_phi [n_r][n_theta] azimuthal block
 * size of each cell's polar block (the coarsening factors c_i of the CFL time
 * step, Sec. 2.3).
 */
MP_API mp_status mp_coarsening_factors(const mp_mesh *mesh, int *c_theta, int *c_phi);

/*
 * Device rate probes (diagnostics, not part of a solve): measures, on the
 * current device, the float64 FMA rate in TFLOP/s (the roofline of the float64
 * path) and the hardware float64 -> float32 conversion rate in conversions/s.
 * Allocates 16 bytes of device memory for the duration of the call.
 */
MP_API mp_status mp_probe_rates(double *fp64_tflops, double *cvt_f64_f32_per_s);

/*
 * Angular moments (step (a), in float64) of rho_dev into ang_dev [n_r][K_L],
 * using the mesh's tables, without allocating any device memory.  The paper
 * has no counterpart: this entry point serves callers that cannot allocate at
 * the point of use -- real-time loops with a memory budget fixed up front, or
 * plug-ins whose host application owns every device allocation.
 * Its only intermediate array lives in a fixed device array of
 * MP_NOALLOC_SCRATCH_DOUBLES float64 values (32 MiB) that every GPU loading
 * this library holds until the process exits; meshes with
 * n_r * n_theta * (2 l_max + 1) above that size, or n_phi above 1536, are
 * rejected with MP_ERR_INVALID_ARG / MP_ERR_UNSUPPORTED before anything runs.
 * The first call on a device looks up that array's device address, so make it
 * before any stream capture.  Work is enqueued on the mesh's stream; calls
 * whose work overlaps on the GPU share the array and race.  rho_dev and
 * ang_dev are device pointers owned by the caller; the moments of the mesh's
 * own solves are not touched.  A NaN or infinite density is recorded in the
 * mesh's device error word and reported as MP_ERR_NONFINITE by the next
 * mp_mesh_synchronize().
 */
#define MP_NOALLOC_SCRATCH_DOUBLES (4u << 20)
MP_API mp_status mp_moments_noalloc(const mp_mesh *mesh, const double *rho_dev, double *ang_dev);

/* Static description of a status code. */
MP_API const char *mp_status_string(mp_status status);

/* Copies the last error detail of this host thread into buf (NUL-terminated). */
MP_API mp_status mp_last_error_detail(char *buf, int len);

/* Library version, as major * 10000 + minor * 100 + patch. */
MP_API int mp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GB300_MULTIPOLE_H */
