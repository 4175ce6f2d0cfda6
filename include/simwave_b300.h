/*
 * simwave_b300.h -- C ABI of the B300 (sm_103a) finite-difference acoustic
 * wave solver.  It implements the method of "simwave - A Finite Difference
 * Simulator for Acoustic Waves Propagation" (arXiv 2201.05278): explicit
 * second-order leapfrog in time (Sec. 2.2, Eq. 6-7), central differences of
 * order 2..20 in space (Sec. 2.3, Eq. 9-10), constant density (Eq. 3) or
 * variable density (Eq. 2 in the expanded form of Eq. 5), an absorbing
 * layer (Sec. 2.1, Eq. 4), null Dirichlet / null Neumann faces, and
 * Kaiser-windowed sinc sources and receivers (Sec. 2.4, Eq. 11-12).
 *
 * Conventions shared by every call
 *   - Axes are (z, y, x) in 3D and (z, x) in 2D; x is contiguous.  Arrays
 *     that describe axes have ndim entries, arrays that describe faces have
 *     2*ndim entries in the order (z-, z+, [y-, y+,] x-, x+).
 *   - Grid-shaped arrays are dense row-major FP32 [nz][ny][nx] (3D) or
 *     [nz][nx] (2D) and include the absorbing layer.
 *   - Array arguments marked "host or device" may point to host memory
 *     (pageable or pinned) or to device memory; the library detects which.
 *     Device memory of the current device (which must be the grid's) and
 *     managed memory are used in place; host memory and device memory of
 *     another GPU go through a buffer of the grid's own.  The caller keeps
 *     ownership of every buffer it passes; input buffers are only read
 *     during the call.
 *   - All device work runs on the stream given to sw_create_grid.
 *   - No call throws; each returns a status.  sw_last_error() returns a
 *     thread-local message for the last failing call of the calling thread.
 *   - A grid handle must not be used from two threads at once.
 */
#ifndef SIMWAVE_B300_H
#define SIMWAVE_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sw_grid sw_grid;
typedef struct sw_batch sw_batch;

typedef enum {
  SW_OK = 0,
  SW_EINVAL = 1,   /* invalid argument (sizes, order, positions, NULL pointers) */
  SW_ECFL = 2,     /* user time step above the stability bound of Eq. 8 */
  SW_ENOMEM = 3,   /* device or host allocation failed */
  SW_ECUDA = 4,    /* a CUDA runtime call failed */
  SW_ETIMEOUT = 5, /* a kernel's bounded wait gave up (device error flag set) */
  SW_ESTATE = 6    /* call out of order (e.g. sw_forward before sw_set_model) */
} sw_status;

enum { SW_BC_NONE = 0, SW_BC_DIRICHLET = 1, SW_BC_NEUMANN = 2 };

/*
 * sw_create_grid -- grid, discretisation, boundary treatment, time step.
 * (Sec. 2.1-2.3, Sec. 4 "SpaceModel"/"TimeModel"; Eq. 4, 8, 9-10.)
 *
 *   out          receives the handle (library-owned; free with sw_destroy_grid)
 *   ndim         2 or 3
 *   shape        [ndim] node counts including the absorbing layer, each >= r+1
 *                where r = space_order/2
 *   spacing      [ndim] grid spacing in metres (> 0)
 *   space_order  even, 2..20 (stencil radius r = space_order/2)
 *   nbl          [2*ndim] absorbing-layer width in cells per face (>= 0); the
 *                physical domain is nodes nbl_lo .. n-1-nbl_hi on each axis
 *   bc           [2*ndim] SW_BC_* per face: Dirichlet holds the face node at
 *                0 with odd ghost mirroring, Neumann mirrors even, NONE uses
 *                zero ghosts
 *   damp_alpha   alpha of eta = alpha d^p (1/s); d is the Euclidean distance
 *                in cells from a node to the physical domain
 *   damp_degree  p >= 0
 *   dt           time step in seconds; <= 0 selects the bound of Eq. 8 once
 *                the velocity is known (sw_set_model).  A positive dt above
 *                that bound makes sw_set_model fail with SW_ECFL.
 *   cuda_stream  cudaStream_t the library enqueues all work on (NULL = the
 *                legacy default stream); the current device at this call is
 *                the grid's device
 * Allocates the two wavefield levels and the model fields on the device.
 */
sw_status sw_create_grid(sw_grid** out, int ndim, const int64_t* shape, const double* spacing,
                         int space_order, const int* nbl, const int* bc, double damp_alpha,
                         int damp_degree, double dt, void* cuda_stream);

/*
 * sw_set_model -- velocity and optional density (Sec. 2, Eq. 2-3, 5).
 *
 *   velocity  grid-shaped FP32, m/s, host or device; every value finite, > 0
 *   density   grid-shaped FP32, any unit, > 0, host or device; NULL selects
 *             the constant-density operator.  With a density the update uses
 *             Lap p - grad(ln rho) . grad p (Eq. 5-7), ln(rho) mirrored even
 *             into the ghost layers.
 * Resolves dt (Eq. 8), builds kappa = (c dt)^2 and the damping coefficients.
 * Returns SW_ECFL if a user dt exceeds the bound.  Synchronises the stream.
 */
sw_status sw_set_model(sw_grid* g, const float* velocity, const float* density);

/*
 * sw_set_acquisition -- sources, receivers, wavelet (Sec. 2.4, Eq. 11-12).
 *
 *   n_src, src_pos      number of sources and their [n_src][ndim] positions
 *                       in metres from the corner of the physical domain
 *                       (host, FP64)
 *   n_rec, rec_pos      same for receivers (host, FP64)
 *   nt, wavelet         [nt] samples S(t_n) shared by every source, or
 *                       [n_src][nt] when wavelet_per_source != 0; FP32, host
 *                       or device
 *   window_radius       Kaiser window half-width r_w, 1..10; every window
 *                       (2 r_w nodes per axis) must lie inside the grid, else
 *                       SW_EINVAL
 * Each point spreads over the nodes with |i - s| < r_w with weights
 * W(i - s) sinc(i - s) per axis (product over axes).
 */
sw_status sw_set_acquisition(sw_grid* g, int n_src, const double* src_pos, int n_rec,
                             const double* rec_pos, int nt, const float* wavelet,
                             int wavelet_per_source, int window_radius);

/*
 * sw_forward -- run n_steps leapfrog steps from rest (p[0] = p[-1] = 0).
 * (Sec. 2.2 Eq. 7, Sec. 3.2 back-end, Sec. 4 "Solver.forward".)
 *
 * Step n (0-based) computes p[n+1] from p[n], p[n-1], adds the sources
 * S(t_n) (t_n = n dt), then records the receivers on p[n+1].
 *   n_steps      >= 0 and <= nt of the acquisition when there are sources
 *   seismogram   [n_steps][n_rec] FP32 output, host or device, may be NULL
 *                when n_rec == 0; row n holds the receivers at t_{n+1}
 *   final_field  grid-shaped FP32 output p[n_steps], host or device, or NULL
 * Synchronises the stream and checks the device error flag before
 * returning (SW_ETIMEOUT if a kernel's bounded wait gave up).
 */
sw_status sw_forward(sw_grid* g, int n_steps, float* seismogram, float* final_field);

/*
 * Misfit gradient by the adjoint-state method.  The paper names full-waveform
 * inversion as the solver's use but prints no adjoint; this is the exact
 * discrete adjoint of the forward recurrence sw_forward runs, with or
 * without density (Eq. 5, Eq. 10).  sw_gradient runs the forward simulation
 * of the current model and acquisition for n_steps, the misfit
 *   J = 1/2 sum_n sum_r (d[n][r] - observed[n][r])^2
 * of its seismogram d against `observed`, and the adjoint sweep backwards in
 * time, and returns J, dJ/dc (the derivative with respect to the velocity
 * at every node) and, with a density model, dJ/drho.
 *   observed         [n_steps][n_rec] FP32, device or host (copied)
 *   misfit           host, one double
 *   grad_vel         [nz][ny][nx] FP32 (2D: [nz][nx]), device or host
 *   grad_rho         same layout, or NULL; needs a density model
 *   checkpoint_every forward states kept every K time steps; each segment
 *                    is recomputed during the adjoint sweep.  K >= n_steps
 *                    keeps every level: the forward run writes p[0] ..
 *                    p[n_steps - 1] into n_steps + 1 padded FP32 fields,
 *                    the sweep recomputes nothing and checkpoint_format
 *                    does not apply (nothing is rounded).  0: every level
 *                    kept when the call's fields fit in 80% of the free
 *                    device memory, else K about sqrt(2 n_steps).
 *   checkpoint_format SW_CKPT_FP32: each checkpoint is a copy of the two
 *                    padded FP32 levels.  16-bit formats keep the nodes of
 *                    p[k0] and of the difference p[k0] - p[k0-1] (small
 *                    next to p; stored on its own, so that the time
 *                    difference a recomputed segment starts from is as
 *                    accurate as the level), so the recomputed segments
 *                    start from rounded states and the gradient carries
 *                    that rounding: SW_CKPT_BF16 / SW_CKPT_FP16 as 16-bit
 *                    floats divided by the field's largest magnitude (one
 *                    scale per snapshot); SW_CKPT_I16 as 16-bit fixed point
 *                    with one scale per (z, y) row of nodes (the rounding
 *                    step is 1/32767 of the row's largest magnitude instead
 *                    of 8 or 11 bits of every value).  Device memory for the call,
 *                    freed before it returns: (2 n_steps / K + K + 4) padded
 *                    FP32 wavefields (K + 4 with 16-bit checkpoints or when
 *                    every level is kept, plus 2 n_steps / K node arrays of
 *                    2 bytes per node with 16-bit checkpoints; 3 or 6 more
 *                    with density) and three [n_steps][n_rec] arrays.
 * Errors: SW_ESTATE before sw_set_model / sw_set_acquisition; SW_EINVAL for
 * grad_rho without a density model, without receivers, for n_steps < 1 or
 * beyond the wavelet, or with 2R+1 nodes or fewer along an axis; SW_ENOMEM
 * when the
 * buffers do not fit.  The grid's wavefields
 * hold the forward run's last two levels afterwards.
 */
enum { SW_CKPT_FP32 = 0, SW_CKPT_BF16 = 1, SW_CKPT_FP16 = 2, SW_CKPT_I16 = 3 };
sw_status sw_gradient(sw_grid* g, int n_steps, const float* observed, double* misfit, float* grad_vel,
                      float* grad_rho, int checkpoint_every, int checkpoint_format);

/*
 * sw_gradient_shots -- the misfit and its gradient summed over several shots
 * (the objective of full-waveform inversion, the use the paper names in
 * Sec. 1 and 6, is a sum over shots; the paper prints no adjoint).  Shot s
 * runs the acquisition's sources moved to its own positions, with the
 * acquisition's receivers and wavelet, against its own observed data; the
 * call returns J = sum_s J_s, dJ/dc = sum_s dJ_s/dc and, with a density
 * model, dJ/drho = sum_s dJ_s/drho.  Each shot runs exactly what
 * sw_gradient runs; the gradient accumulators, checkpoints and segment
 * buffers are allocated once for all shots, and the velocity gradient is
 * formed once from the summed accumulator.
 *   n_shots          >= 1
 *   shot_src_pos     host FP64 [n_shots][n_src][ndim]: every shot's source
 *                    positions (metres, as in sw_set_acquisition; n_src is
 *                    the acquisition's source count, >= 1); all windows are
 *                    checked before any device work
 *   observed         [n_shots][n_steps][n_rec] FP32, device or host
 *   misfit, grad_vel, grad_rho, checkpoint_every, checkpoint_format: as in
 *                    sw_gradient (the sums over the shots)
 * The acquisition keeps its own source positions afterwards.  Device memory
 * as one sw_gradient call.  Errors: as sw_gradient; SW_EINVAL for
 * n_shots < 1, NULL positions, an acquisition without sources or a shot
 * window that leaves the grid.
 */
sw_status sw_gradient_shots(sw_grid* g, int n_shots, const double* shot_src_pos, int n_steps, const float* observed,
                            double* misfit, float* grad_vel, float* grad_rho, int checkpoint_every,
                            int checkpoint_format);

/*
 * Memory-capped schedule for sw_gradient: with max_states = s > 0 the adjoint
 * sweep keeps at most s forward states (pairs of padded FP32 levels) besides
 * two working levels and follows the binomial checkpointing schedule (the
 * recursive form of Griewank's revolve): after a plain forward run for the
 * residuals, steps (l, r] are reversed by storing the state at
 * m = r - min(C(s - 1 + t, s - 1), r - l - 1), t the least count with
 * C(s + t, s) >= r - l, reversing (m, r] with one slot fewer and then (l, m].
 * Device memory: 2 s + 5 padded fields (+3 or 6 with density) instead of the
 * uniform scheme's 2 n_steps / K + K + 4; the forward steps recomputed grow
 * like n_steps times the least t.  The gradient is the same as with uniform
 * checkpoints.  0 (the default) selects the uniform segments of
 * checkpoint_every steps.  Needs checkpoint_format SW_CKPT_FP32 (SW_EINVAL
 * from sw_gradient otherwise).  Errors: SW_EINVAL for a negative budget.
 */
sw_status sw_set_checkpoint_budget(sw_grid* g, int max_states);

/*
 * sw_get_dt -- the time step in use, in seconds (Sec. 2.2, Eq. 8).
 *   dt  host, one double: the user's dt, or after sw_set_model with an
 *       automatic dt (<= 0 at sw_create_grid) the stability bound of Eq. 8,
 *       dt = 2 / (c_max sqrt(sum_axes a / h^2)), a = |v_0| + 2 sum_j |v_j|
 * Errors: SW_EINVAL for NULL arguments; SW_ESTATE when the time step is
 * automatic and no model is set yet.
 */
sw_status sw_get_dt(const sw_grid* g, double* dt);

/*
 * Ricker wavelet samples, host-side helper (Sec. 2.4, default wavelet):
 * out[n] = (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), tau = n dt - t0,
 * computed in FP64 and rounded to FP32.  out is host memory [nt].
 */
sw_status sw_ricker(double f_peak, double t0, double dt, int nt, float* out);

/*
 * Stencil kernel variant.  CUDA implementations of the same update (Eq. 7):
 * SW_STENCIL_AUTO picks the TMA-pipelined persistent kernel for 3D grids
 * (constant or variable density), the cluster-resident run for 2D grids that
 * fit it, the two-step kernel (below) for other 2D grids of constant density
 * with 4M nodes or more, and the per-step plain kernels otherwise; SW_STENCIL_PLAIN forces the
 * per-step plain kernels; SW_STENCIL_TMA asks for the pipelined kernel (3D
 * only, else SW_EINVAL; cases it does not cover still use the plain
 * kernel).  SW_STENCIL_CLUSTER asks for the cluster-resident run (2D only,
 * else SW_EINVAL): the whole forward run in one launch of one thread-block
 * cluster (up to 16 CTAs, one per SM) whose shared memory holds both
 * levels and kappa, for 2D grids of constant density whose rows fit (two
 * levels of ceil(nz / C) + 2R rows of nx + 2R floats plus ceil(nz / C) rows
 * of kappa per CTA, at most the device's per-block shared memory), without
 * distributed forcing or snapshot frames; other cases use the plain
 * kernels.  It gives the same values as the plain 2D kernels bit for bit.
 * SW_STENCIL_TB2 asks for temporal blocking (2D only, else SW_EINVAL): two
 * leapfrog steps per launch, each tile staging p[n] with a 2R ring and
 * p[n-1], kappa with an R ring in shared memory, computing p[n+1] on the
 * tile and its ring (step n's sources and the face images included) and
 * p[n+2] on the tile, then a face pass per new level (ghosts, receivers)
 * with step n+1's sources in between; 20 bytes of memory traffic per two
 * node updates instead of 32.  For 2D grids of constant density without
 * distributed forcing or snapshot frames (others use the plain kernels);
 * an odd last step runs on the plain kernels; the grid allocates two more
 * wavefield levels on its first such run.  The levels equal the plain
 * kernels' bit for bit when no two source taps share a node (the
 * seismograms agree to rounding: another receiver sampler).  SW_STENCIL_AUTO
 * picks it for such 2D grids of 4M nodes or more (where it is faster than
 * the per-step kernels; below, their fields stay in L2 and it is slower).
 * sw_get_stencil_variant reports the kernel sw_forward will launch for the
 * current model.
 */
enum { SW_STENCIL_AUTO = 0, SW_STENCIL_PLAIN = 1, SW_STENCIL_TMA = 2, SW_STENCIL_CLUSTER = 3, SW_STENCIL_TB2 = 4 };
sw_status sw_set_stencil_variant(sw_grid* g, int variant);
sw_status sw_get_stencil_variant(const sw_grid* g, int* variant);

/*
 * Distributed forcing (the forcing term of Eq. 5, used by the manufactured
 * solutions of Sec. 2.5): every later sw_forward adds
 * f(x, t_n) = sum_m F_m(x) T_m(t_n) at step n the way a source enters Eq. 7,
 * p[n+1] += kappa a f, except at Dirichlet face nodes.  fields is
 * [n_force][nodes] (dense, (z, [y,] x) order, the grid's full shape),
 * signatures is [n_force][n_sig] (T_m at t_n = n dt); both FP32, host or
 * device, copied (the caller keeps ownership).  n_force = 0 removes the
 * forcing.  A later sw_forward longer than n_sig steps fails with SW_EINVAL.
 * Errors: SW_EINVAL for NULL arrays or n_sig < 1 with n_force > 0,
 * SW_ENOMEM.
 */
sw_status sw_set_forcing(sw_grid* g, int n_force, const float* fields, const float* signatures, int n_sig);

/*
 * Initial levels p[0] = p0 and p[-1] = pm1 of every later sw_forward (dense
 * [nodes] FP32, host or device, copied; NULL = zero, the default).  This
 * resumes a run from a saved pair of levels (two are needed, Eq. 7) and sets
 * up standing-wave tests.  Dirichlet face nodes are taken as 0 and the ghost
 * nodes follow the face conditions.  Errors: SW_ENOMEM.  sw_gradient
 * refuses to run (SW_ESTATE) while initial levels or forcing are set.
 */
sw_status sw_set_initial_state(sw_grid* g, const float* p0, const float* pm1);

/*
 * Wavefield snapshots (the solver's saving stride, Sec. 4): with
 * saving_stride = s > 0, every later sw_forward writes p after s, 2s, 3s, ...
 * time steps into consecutive frames of `snapshots` (frame k = p after
 * (k+1) s steps, laid out like final_field), stopping after max_frames
 * frames; s = 1 saves every step.  s = 0 turns saving off (the last level is
 * still available through sw_forward's final_field).  `snapshots` is
 * caller-owned device memory of max_frames x (nodes) floats; the grid only
 * keeps the pointer.  Errors: SW_EINVAL for a negative stride or count, a
 * missing or host buffer with s > 0.
 */
sw_status sw_set_saving(sw_grid* g, int saving_stride, float* snapshots, int64_t max_frames);

/*
 * Batched shots.  The paper's solver runs one shot at a time; waveform
 * inversion, the use it names (Sec. 1 and 6), runs many shots.  A batch
 * advances several 2D constant-density grids (one space order, one device
 * and stream, any sizes) together: per time step one stencil launch over a
 * work list of (model, tile) for all shots, one injection and one receiver
 * launch.  Grids of the same geometry (shape, spacing, absorbing layers,
 * faces, damping, dt) whose kappa fields are bit-identical are one model
 * group: each tile of the model is read once per step for all its shots.
 * Every shot gives the same result as sw_forward on its grid alone.
 *
 * A batch of 3D constant-density grids (any sizes, one space order, every
 * grid with equal spacings along its axes or none) runs per time step one
 * launch of the pipelined stencil over a work list of (64 x 16 tile, plane)
 * items of all grids, and one launch of every grid's face conditions,
 * receiver samples and next step's sources (which enter through the level
 * the step reads as p[n-1], as in sw_forward); small grids, which alone
 * leave most of the GPU idle or pay a warm-up per tile column, share the
 * launch.  Each grid gives the same result as sw_forward on it alone, bit
 * for bit.
 *
 * sw_create_batch borrows the grids (they must outlive the batch and keep
 * their model and acquisition; a grid changed afterwards makes
 * sw_batch_forward fail with SW_ESTATE).  Errors: SW_EINVAL for
 * variable-density grids, grids of different dimensions, mixed orders,
 * streams or devices, a grid listed twice, grids with forcing or snapshots,
 * and (3D) grids the pipelined kernel does not take (sw_set_stencil_variant
 * plain, too large), mixed equal and unequal spacings, or source windows
 * where eta dt reaches 1/2; SW_ESTATE for a grid without model or
 * acquisition.
 *
 * sw_batch_forward runs n_steps steps of every grid from rest (or from its
 * sw_set_initial_state levels).  seismograms[i] is grid i's [n_steps][n_rec]
 * output in DEVICE memory (may be NULL for grids without receivers);
 * final_fields (NULL, or an array with NULL entries to skip) receives p
 * after the last step (host or device).  The time loop is captured as a CUDA
 * graph on the second call with the same n_steps.  Blocks until done.
 *
 * sw_batch_info: number of model groups (3D: grids) and of work items
 * (tile of one shot; 3D: tile and plane) per step.
 *
 * Tile shape (2D): tiles are 128 columns wide and 16, 32 or 64 rows high.
 * sw_create_batch tunes the height on the batch itself: it times a few
 * stencil launches with each height (on zeroed fields) and keeps the
 * fastest.  sw_batch_get_tile returns the height in use and, if tuned_us is
 * not NULL, the three timings (microseconds per launch, heights 16, 32, 64);
 * sw_batch_set_tile forces a height (SW_EINVAL for another value, and for
 * a 3D batch, whose tiles are those of the pipelined kernel).  The results
 * do not depend on the height.
 * sw_batch_set_profiling / sw_batch_get_profile: as for a grid (every
 * every-th stencil launch timed with CUDA events).
 */
sw_status sw_create_batch(sw_batch** out, sw_grid* const* grids, int n_grids);
sw_status sw_batch_forward(sw_batch* b, int n_steps, float* const* seismograms, float* const* final_fields);
sw_status sw_batch_info(const sw_batch* b, int* n_groups, int* n_items);
sw_status sw_batch_get_tile(const sw_batch* b, int* tile_rows, float* tuned_us);
sw_status sw_batch_set_tile(sw_batch* b, int tile_rows);
sw_status sw_batch_set_profiling(sw_batch* b, int every);
sw_status sw_batch_get_profile(const sw_batch* b, double* stencil_ms, int64_t* stencil_launches,
                               int64_t* kernel_launches);
void sw_destroy_batch(sw_batch* b);

/*
 * Failure-path test hook (no counterpart in the paper).  With starve != 0
 * the TMA-pipelined kernel issues no tensor copies, so every mbarrier wait
 * in it runs into its bound: the kernel raises the device error flag and
 * returns, and sw_forward reports SW_ETIMEOUT with the CUDA context intact.
 * wait_limit_ns bounds each wait (0 restores the default of 2 s); it also
 * applies with starve = 0.  Nothing faults or hangs: the test only shows
 * that a stalled pipeline ends with an error status.
 */
sw_status sw_set_pipeline_test(sw_grid* g, int starve, unsigned long long wait_limit_ns);

/*
 * Kernel timing.  With every = N > 0, sw_forward records CUDA events around
 * every N-th stencil launch (time steps 0, N, 2N, ...) on the grid's stream
 * (N = 1: all of them; a sample keeps the events' own cost out of the run);
 * every = 0 turns timing off.  sw_get_profile returns, for the last
 * sw_forward, the summed time of the timed stencil launches, how many were
 * timed, and the number of kernels it launched in total (after sw_gradient:
 * no timed launches, and the kernels that call launched).  A 2D run on the
 * cluster-resident kernel (SW_STENCIL_CLUSTER) is one launch for all time
 * steps: with timing on, its time is reported with n_steps timed launches,
 * so that the time per launch is the time per step.
 */
sw_status sw_set_profiling(sw_grid* g, int every);
sw_status sw_get_profile(const sw_grid* g, double* stencil_ms, int64_t* stencil_launches,
                         int64_t* kernel_launches);

/* Bytes of device memory the grid holds (wavefields, model, acquisition). */
sw_status sw_get_device_bytes(const sw_grid* g, int64_t* bytes);

/*
 * sw_forward_noalloc -- the whole forward run of sw_create_grid +
 * sw_set_model + sw_set_acquisition + sw_forward in one call that allocates
 * no device memory.  The paper has no counterpart; it exists for callers that
 * cannot call cudaMalloc: programs whose device memory belongs to a pool or
 * framework allocator with a fixed budget, and loops that cannot afford the
 * device-wide synchronisation cudaMalloc/cudaFree imply.
 *
 * Arguments mean what they mean in the four calls above, with these limits:
 *   - velocity, density (NULL for constant density), seismogram and
 *     final_field (NULL to skip) must be plain device memory (not managed)
 *     of the current device, else SW_EINVAL; positions are host memory; the
 *     wavelet may be host memory or device memory of the current device.
 *     The library cannot see buffer sizes: velocity, density and final_field
 *     hold the grid's node count, the seismogram n_steps * n_rec values and
 *     the wavelet nt (or n_src * nt) samples.
 *   - Wavefields, model fields, damping table and window weights live in one
 *     static device array of SW_NOALLOC_SCRATCH_BYTES that every GPU which
 *     loads the library holds until the process exits.  A problem that needs
 *     more (about three padded FP32 copies of the grid, four with density),
 *     or a grid of more than 2^34 nodes, is rejected with SW_EINVAL before
 *     any device work; the message gives the bytes needed.
 *   - Every call looks up the array's device address (cudaGetSymbolAddress,
 *     which allocates nothing) with the caller's device current.  The first
 *     lookup on a device may load the library's device code, so make the
 *     first call on a device before any stream capture on it.
 *   - Every call shares the same array and leaves its contents behind (the
 *     call clears what must start at zero).  Calls whose GPU work overlaps,
 *     on one device, race on the array and give wrong results: serialise them.
 *   - It always runs the plain per-step kernels (stencil, then source
 *     injection and receiver sampling as separate launches), not the
 *     pipelined 3D kernel or the cluster-resident 2D run that sw_forward
 *     picks: its results match sw_forward's within the FP32 parity
 *     tolerance, not bit for bit, and it runs slower.
 *   - Synchronises the stream before returning, like sw_forward.
 */
#define SW_NOALLOC_SCRATCH_BYTES (32ull << 20)
sw_status sw_forward_noalloc(int ndim, const int64_t* shape, const double* spacing, int space_order,
                             const int* nbl, const int* bc, double damp_alpha, int damp_degree,
                             double dt, const float* velocity, const float* density, int n_src,
                             const double* src_pos, int n_rec, const double* rec_pos, int nt,
                             const float* wavelet, int wavelet_per_source, int window_radius,
                             int n_steps, float* seismogram, float* final_field, void* cuda_stream);

/* Message describing the last failing call on this thread ("" if none). */
const char* sw_last_error(void);

/* Frees the handle and its device memory (NULL is accepted). */
void sw_destroy_grid(sw_grid* g);

#ifdef __cplusplus
}
#endif

#endif /* SIMWAVE_B300_H */
