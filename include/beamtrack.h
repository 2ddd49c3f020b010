/*
 * beamtrack.h - C ABI of the B300-native space-charge tracking step.
 *
 * One s-step of ImpactX-style beam tracking (arXiv:2208.02382, section
 * "ImpactX" and its subsection "Model Assumptions"): macroparticles in 6D
 * phase space relative to a reference particle are pushed through linear
 * symplectic element maps, and space charge enters as a split-operator kick:
 * charge deposition to a 3D grid in the bunch rest frame, an open-boundary
 * Poisson solve, field gather and momentum kick.  The paper prints no
 * formulas; each call below names the reading it implements.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Phase space (x, px, y, py, t, pt): x, y [m]; px, py = transverse momentum
 *   over the reference momentum; t = c * (arrival-time lag) [m];
 *   pt = -(energy deviation) / (reference momentum * c).
 * - Particle data are six device arrays of n doubles (structure of arrays),
 *   owned by the caller.  The library never allocates, frees or keeps
 *   particle memory; it may reorder particles (all six arrays and `id`
 *   together) to bin them by grid cell.
 * - Grid arrays are owned by the caller; node (i, j, l) of an N^3 grid sits at
 *   flat index i + N*(j + N*l) (x fastest).
 * - Rest frame: X = x, Y = y, Z = -beta*gamma*t (Model Assumptions: linear
 *   boost of the reference particle).
 * - Every call is asynchronous on `stream` (a cudaStream_t, or NULL for the
 *   legacy default stream) unless stated.  Argument errors are detected on
 *   the host before any launch and returned at once; device-side errors
 *   (a non-finite coordinate, a particle outside a given box) are recorded in a
 *   device status word and returned by the next call that reads it
 *   (bx_sync, bx_moments) or by bx_sync.
 * - Status codes are the BX_* values below; bx_last_error() gives text.
 * - No call throws; no C++ exception crosses this ABI.
 */
#ifndef BEAMTRACK_H
#define BEAMTRACK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define BX_OK 0
#define BX_BAD_ARG 1        /* null pointer, size out of range, bad element */
#define BX_NONFINITE 2      /* NaN or Inf found in particle coordinates     */
#define BX_OUT_OF_MEMORY 3  /* a device allocation of the context failed    */
#define BX_DEVICE_TIMEOUT 4 /* a device-side wait ran past its time limit: the
                             moments' staged copies (2 s per wait), reported
                             by bx_sync; bx_selftest_wait_timeout makes one */
#define BX_CUDA 5           /* a CUDA runtime call failed                   */
#define BX_COLLECTIVE 6     /* a sharded run's allreduce callback failed    */

/* ---- element types (Listing 1: elements.Drift, elements.Quad; sector bend
 *      from the paper's chicane benchmark; thin dipole edge and constant
 *      focusing from its list of benchmarks) ---------------------------------- */
#define BX_DRIFT 0
#define BX_QUAD 1
#define BX_SBEND 2
#define BX_DIPEDGE 3 /* thin: nslice = 0, angle = edge angle, k = curvature 1/rho */
#define BX_CONSTF 4  /* constant focusing: k = k_x, k2 = k_y [1/m^2]            */
#define BX_MULTIPOLE 5 /* thin: nslice = 0, order m, k = kn, k2 = ks [1/m^(m-1)] */
#define BX_MULTIPOLE_MAX_ORDER 12

typedef struct bx_ctx bx_ctx;
typedef struct bx_batch bx_batch;

/* Options of a context.
 * n_grid         : nodes per dimension N of the charge/potential grid; a power
 *                  of two in [8, 256].  The Poisson solve runs on the doubled
 *                  (2N)^3 grid.
 * shape_order    : particle shape (Listing 1 set_particle_shape): 1 (CIC) or
 *                  2 (TSC).
 * rebin_interval : kicks between re-binning the particles by grid bin (a
 *                  stable counting sort that keeps the deposit's shared-memory
 *                  tiles compact), counted on the context's kick counter (it
 *                  carries over between bx_track calls until bx_reset): 0 =
 *                  default (16), -1 = never, else >= 1.
 * bin_edge       : grid cells per bin edge: 0 = default (8, or N/16 above
 *                  N = 128), else a power of two in [2, N/2] with at most 16^3
 *                  bins.
 * cell_order     : 0 = re-bin by bin only; 1 = by bin and, within a bin, by
 *                  grid cell (a second counting-sort pass), so that consecutive
 *                  particles share field nodes in the gather's loads.  None of
 *                  the three changes any result, only the speed
 *                  (bx_autotune_binning picks them by timing).
 */
typedef struct {
    int32_t n_grid;
    int32_t shape_order;
    int32_t rebin_interval;
    int32_t bin_edge;
    int32_t cell_order;
    int32_t reserved[3];
} bx_options;

/* A bunch.  coord[0..5] = x, px, y, py, t, pt: device pointers to n doubles
 * each, 8-byte aligned.  id: device pointer to n int64 ids, or NULL (then
 * particles are not reordered).  charge_sign: +1 or -1 (species);
 * bunch_charge_C: |Q| of the whole bunch [C] (Listing 1 add_particles);
 * mass_MeV, kinetic_MeV: reference particle rest and kinetic energy
 * (Listing 1 set_energy_MeV, read as kinetic).  n may be 0. */
typedef struct {
    double *coord[6];
    int64_t *id;
    int64_t n;
    double charge_sign;
    double bunch_charge_C;
    double mass_MeV;
    double kinetic_MeV;
} bx_beam;

/* One lattice element (Listing 1: Drift(ds, nslice), Quad(ds, k, nslice)).
 * Thick elements (drift, quadrupole, sector bend, constant focusing): length
 * [m] > 0; nslice >= 1 slices, one space-charge kick per slice; k [1/m^2]
 * (quadrupole: k > 0 focuses x; constant focusing: k_x); angle [rad] (sector
 * bend, total over the element); k2 [1/m^2] (constant focusing: k_y).
 * Thin dipole edge (hard-edge fringe field, K. L. Brown SLAC-75: px += h
 * tan(psi) x, py -= h tan(psi) y): nslice = 0, angle = edge angle psi, k =
 * curvature h = 1/rho of the bend it belongs to; it takes no kick and acts
 * between the slices around it (a rectangular bend of angle theta: edges of
 * theta/2 on both faces).  Thin multipole (paper: a chain of thin multipoles;
 * the kick is the reading dpx - i dpy = -(kn + i ks) (x + i y)^(m-1)/(m-1)!
 * of a straight 2D multipole magnet, so m = 2 with kn > 0 focuses x like a
 * quadrupole with k > 0): nslice = 0, order = m in 1..BX_MULTIPOLE_MAX_ORDER
 * (1 dipole, 2 quadrupole, 3 sextupole, ...), k = kn, k2 = ks (integrated
 * strengths); x, y, t, pt are unchanged.  Thin elements ahead of slice j act
 * in the call that tracks slice j; those after the last slice act at the end
 * of the call that tracks it.  order is ignored by the other element types. */
typedef struct {
    int32_t type;
    int32_t nslice;
    double length;
    double k;
    double angle;
    double k2;
    int32_t order;
    int32_t reserved;
} bx_element;

/* A lattice in HOST memory.  space_charge: 0 = maps only
 * (Listing 1 set_space_charge(False)), 1 = split-operator kicks. */
typedef struct {
    const bx_element *elements;
    int32_t count;
    int32_t space_charge;
} bx_lattice;

/* A grid.  n must equal the context's n_grid.
 * use_box = 1: the box [lo, hi) given here is used as is;
 * use_box = 0: the context's box rule is applied (see bx_deposit) and the
 *              chosen box is written back to lo/hi/h.
 * h = (hi - lo)/(n - 1) per dimension (output).
 * rho: device, n^3 doubles [C/m^3].  phi: device, (n+2)^3 doubles [V],
 * holding nodes -1..n per dimension (array index k = node k - 1). */
typedef struct {
    int32_t n;
    int32_t use_box;
    double lo[3];
    double hi[3];
    double h[3];
    double *rho;
    double *phi;
} bx_grid;

/* Create a context on the current CUDA device.  The context owns its device
 * scratch (fixed-point charge accumulators, FFT work buffers, the Green's
 * function spectrum, reduction buffers, status word); it holds the grid box
 * and the kick counter between calls.  Returns BX_BAD_ARG for a bad n_grid or
 * shape_order, BX_OUT_OF_MEMORY / BX_CUDA on allocation failure. */
int32_t bx_create(bx_ctx **out, const bx_options *opt);

/* Destroy a context (synchronises the device first).  NULL is allowed. */
int32_t bx_destroy(bx_ctx *ctx);

/* Forget the box, the Green's function, the kick counter and the regrid log. */
int32_t bx_reset(bx_ctx *ctx);

/* Track the bunch through slices [first_kick, first_kick + nkicks) of the
 * lattice's slice schedule (Listing 1 sim.evolve(); Model Assumptions:
 * map-based split-operator step).  Reading: each slice of length
 * ds = length/nslice is map(ds/2), space-charge kick over ds, map(ds/2);
 * adjacent half-maps inside one call are merged into one map.  Before each
 * kick the box rule runs: regrid when a particle lies outside [lo, hi) or an
 * extent fell below half the box; the new box is centred on the bunch with
 * half-width 0.55 * extent; the Green's function is rebuilt when h changes.
 * The bunch is left at a slice boundary.  nkicks = -1 tracks to the end.
 * Each kick's solve is the one of bx_solve computed in block floating point
 * (int64 values, one exponent per FFT line; its kicks agree with an FP64
 * solve's to about 1e-14 of their size).
 * BX_BAD_ARG if first_kick/nkicks fall outside the schedule or an element is
 * invalid.  Non-finite coordinates are reported as BX_NONFINITE by bx_sync. */
int32_t bx_track(bx_ctx *ctx, bx_beam *beam, const bx_lattice *lattice,
                 int64_t first_kick, int64_t nkicks, void *stream);

/* bx_track that also writes the beam moments at the end of every slice
 * (Listing 1 set_slice_step_diagnostics) to moments_device: nkicks x 27
 * doubles in the layout of bx_moments (means, then the centred second
 * moments), entry k for the end of slice first_kick + k.  The moments after
 * each kick are taken back to the slice end through the inverse of the next
 * half map (linear maps carry moments exactly).  Launches each kick's kernels
 * one by one.  BX_BAD_ARG for an empty beam. */
int32_t bx_track_diagnostics(bx_ctx *ctx, bx_beam *beam, const bx_lattice *lattice,
                             int64_t first_kick, int64_t nkicks, double *moments_device,
                             void *stream);

/* Initial bunch in the parametrisation of Listing 1 (distribution.Waterbag):
 * params (host, 9) = {sigmaX, sigmaY, sigmaT, sigmaPx, sigmaPy, sigmaPt,
 * muxpx, muypy, mutpt}.  Per plane, from unit-rms uncorrelated (a, b):
 * u = sigmaU/sqrt(1-mu^2) a, pu = sigmaPu (b - mu/sqrt(1-mu^2) a) (reading:
 * rms u = sigmaU/sqrt(1-mu^2), correlation -mu).  kind 0 (Gaussian): (a, b)
 * are the normals.  kind 1 (Waterbag, uniform in a 6D ball of unit rms per
 * coordinate): the direction of the six normals times sqrt(8) u^(1/6).
 * normals: six device arrays of n standard-normal draws; uniforms: device
 * array of n draws in [0, 1) (kind 1; may be NULL for kind 0); out: six device
 * arrays of n.  BX_BAD_ARG for |mu| >= 1 or an unknown kind; errors via
 * bx_last_error(NULL).  Asynchronous. */
int32_t bx_distribution_beam(int32_t kind, const double params[9],
                             const double *const normals[6], const double *uniforms, int64_t n,
                             double *const out[6], void *stream);

/* Charge deposition (ABLASTR charge deposition reused by ImpactX; Listing 1
 * particle shape 1 = CIC): rho[node] = q * sum_p wx*wy*wz / (hx*hy*hz) over
 * the 8 nodes of each particle's cell, q = charge_sign*bunch_charge_C/n,
 * u = (X - lo)/h, i = floor(u) clamped to [0, n-2], weights (1-f, f).
 * With grid->use_box = 0 the context's box rule picks (and remembers) the
 * box.  The result does not depend on particle order (fixed-point
 * accumulation). */
int32_t bx_deposit(bx_ctx *ctx, const bx_beam *beam, bx_grid *grid, void *stream);

/* Open-boundary Poisson solve in the rest frame (Model Assumptions; ABLASTR
 * Poisson solve): phi = G (*) rho as the aperiodic convolution computed on the
 * zero-padded (2n)^3 grid by FFT (Hockney), with G the cell-integrated
 * Green's function (Qiang et al. 2006) built in double-double precision for
 * the grid's h; FFTs in FP64.  Reads grid->rho and grid->h, writes grid->phi
 * on nodes -1..n. */
int32_t bx_solve(bx_ctx *ctx, bx_grid *grid, void *stream);

/* Field gather and momentum kick over a slice ds > 0 (Model Assumptions:
 * electrostatic rest-frame field).  E = -grad phi by centred differences on
 * the nodes, interpolated with the same CIC weights as the deposit, then
 * dpx = s*Ex*ds/(mc^2[eV]*(beta gamma)^2), dpy likewise,
 * dpt = -s*Ez*ds/(mc^2[eV]*beta gamma).  Uses grid->lo/h and grid->phi. */
int32_t bx_gather_kick(bx_ctx *ctx, bx_beam *beam, const bx_grid *grid, double ds,
                       void *stream);

/* Beam statistics (ABLASTR beam statistics; FODO/IOTA benchmarks check second
 * moments): out_device[0..5] = means, out_device[6..26] = the 21 centred
 * second moments in row-major upper-triangle order (00,01,..,05,11,..,55).
 * Two passes over the particles: each coordinate's exact extent, then exact
 * integer sums of the coordinates rounded at 2^-43 of that extent (relative to
 * its rounded midpoint) and of their 21 pairwise products, added in 128-bit
 * integers and converted once.  Every sum is exact, so the result does not
 * depend on particle order (bitwise reproducible for a given set of
 * particles).  The second pass stages the particles in shared memory with bulk
 * asynchronous copies when all six arrays are 16-byte aligned (plain loads
 * otherwise); each wait for a copy is bounded (2 s), and one that runs out
 * records BX_DEVICE_TIMEOUT for the next bx_sync.  All 27 are NaN when a
 * coordinate is not finite or a wait ran out. */
int32_t bx_moments(bx_ctx *ctx, const bx_beam *beam, double *out_device, void *stream);

/* Self-test of that bounded device wait: one block arms a barrier for copies
 * that are never issued, waits on it for limit_ms (0 < limit_ms <= 10000)
 * exactly as the moments' staging waits, gives up and records the timeout in
 * the context's status word.  The next bx_sync returns BX_DEVICE_TIMEOUT (and
 * clears it); the context stays usable.  Nothing faults or hangs. */
int32_t bx_selftest_wait_timeout(bx_ctx *ctx, double limit_ms, void *stream);

/* Integrated Green's function table used by bx_solve: out_device receives
 * (n+1)^3 doubles G[(c*(n+1) + b)*(n+1) + a] for offsets a, b, c = 0..n cells
 * at cell size h[3] [m], in V*m^3/C (the potential at the origin per unit
 * charge density filling the cell at that offset). */
int32_t bx_green_table(bx_ctx *ctx, const double h[3], double *out_device, void *stream);

/* Copy up to `cap` entries of the regrid log (kick indices, counted from the
 * context's creation or last reset, where the box rule made a new box) into
 * host memory; *count receives the total number logged.  Synchronous. */
int32_t bx_regrid_log(bx_ctx *ctx, int64_t *out_host, int64_t cap, int64_t *count);

/* The current box (host copy; synchronous).  Returns BX_BAD_ARG if no box yet. */
int32_t bx_get_box(bx_ctx *ctx, double lo[3], double hi[3], double h[3]);

/* Kernel-level profiling (the paper's ABLASTR layer lists profiling among its
 * reused routines).  Every kernel launch of this context is counted per
 * kernel; with timing = 1 each launch is also bracketed by a pair of CUDA
 * events on its stream.  bx_profile resets counts and times. */
int32_t bx_profile(bx_ctx *ctx, int32_t timing);

/* Read the profile (synchronous: waits for the recorded events).  ms[k] and
 * launches[k] receive the summed device time and the launch count of kernel
 * k for k < min(cap, *count); *count receives the number of kernel kinds.
 * Either array may be NULL. */
int32_t bx_profile_read(bx_ctx *ctx, double *ms, int64_t *launches, int32_t cap,
                        int32_t *count);

/* Name of kernel kind `id` (0 <= id < count of bx_profile_read), or "". */
const char *bx_kernel_name(int32_t id);

/* Charge deposition that allocates nothing, for callers that may not
 * allocate device memory once they are running (for example an on-line model
 * in an accelerator control loop with a fixed memory footprint, or a host
 * framework that owns all device memory through its own pool).  The paper has
 * no counterpart.  It is the arithmetic of bx_deposit with use_box = 1 (the
 * same cells, fixed-point weights and accumulation: bitwise the same rho) and
 * needs no context.
 * beam: as for bx_deposit (device arrays); lo, hi: host arrays, the box;
 * n: nodes per dimension, a power of two in [8, 64]; rho: device output of
 * n^3 doubles.  flags_device: NULL, or a device int32 owned by the caller into
 * which the call ORs BX_NOALLOC_OUTSIDE when particles lay outside the box and
 * BX_NOALLOC_NONFINITE when a position was NaN or Inf; such particles are
 * skipped (their charge is missing from rho).  The caller clears the word.
 * Scratch: the fixed-point accumulators live in one static device array of
 * 2 x 64^3 x 8 bytes = 4 MiB that the library holds on every GPU that loads
 * it until the process exits; n > 64 is rejected with BX_BAD_ARG.  Every call
 * on a device shares that array and clears it first, so calls that overlap on
 * the GPU race: order them on one stream.  The first call on a device looks up
 * the array's device address with that device current and caches it; make
 * that first call before any stream capture.  Asynchronous on `stream`;
 * argument errors are returned at once and described by bx_last_error(NULL). */
#define BX_NOALLOC_OUTSIDE 1
#define BX_NOALLOC_NONFINITE 2
int32_t bx_deposit_noalloc(const bx_beam *beam, const double lo[3], const double hi[3],
                           int32_t n, double *rho, int32_t *flags_device, void *stream);

/* ---- Differentiation (reverse mode) ------------------------------------
 * The paper motivates coupling the code to machine-learning workflows
 * (Introduction, Outlook) but gives no adjoint.  These calls give the
 * gradient of L = w[0] eps_x + w[1] eps_y + w[2] sigma_x + w[3] sigma_y of
 * the bunch after a whole lattice (eps = unnormalised rms emittance
 * sqrt(<du^2><dpu^2> - <du dpu>^2), sigma = rms size) with respect to every
 * element's quadrupole strength k and to the initial coordinates, by a
 * hand-written reverse of each kernel (map transpose, scatter of the kick
 * adjoint, the transposed field stencil, the same Green's convolution, the
 * deposit's weight derivative) with step checkpointing and recomputation.
 * Reading: the grid box is piecewise constant in the coordinates (it changes
 * only at a regrid) and is held fixed: the gradient is the exact derivative
 * of tracking with the run's box sequence replayed (box_replay below). */

/* Twiss-parametrised bunch (Courant-Snyder): for each transverse plane
 * u = sqrt(eps*beta)*xi_u, pu = sqrt(eps/beta)*(xi_pu - alpha*xi_u);
 * t = sigma_t*xi_t, pt = sigma_pt*xi_pt.  twiss (host) = {alpha_x, beta_x,
 * eps_x, alpha_y, beta_y, eps_y, sigma_t, sigma_pt}; xi: six device arrays of
 * n standard-normal draws (x, px, y, py, t, pt order); out: six device arrays
 * of n doubles (may be the beam's).  BX_BAD_ARG for beta <= 0, eps < 0 or
 * non-finite parameters; errors via bx_last_error(NULL).  Asynchronous. */
int32_t bx_twiss_beam(const double twiss[8], const double *const xi[6], int64_t n,
                      double *const out[6], void *stream);

/* dL/d(alpha_x, beta_x, eps_x, alpha_y, beta_y, eps_y) (out, host) from
 * S[i*6 + j] = sum_p dL/dz0_i * z0_j (bx_grad_backward's S_out) by the chain
 * rule through bx_twiss_beam: du/dbeta = u/(2 beta), dpu/dbeta = -pu/(2 beta),
 * du/deps = u/(2 eps), dpu/deps = pu/(2 eps), dpu/dalpha = -u/beta. */
int32_t bx_twiss_grad(const double twiss[8], const double S[36], double out[6]);

/* The objectives of the differentiation calls from the 27 moments of
 * bx_moments (host copy): out = (eps_x, eps_y, sigma_x, sigma_y), eps =
 * sqrt(<du^2><dpu^2> - <du dpu>^2) (unnormalised rms emittance), sigma =
 * sqrt(<du^2>).  BX_NONFINITE if one is not a finite number.  Host only. */
int32_t bx_objectives(const double moments[27], double out[4]);

/* Chain rule for quadrupole strengths shared by several elements: dk_family[f]
 * = sum of dk_element[e] over the elements e with family[e] = f (host arrays;
 * family[e] = -1: the element's strength is not a parameter).  BX_BAD_ARG for
 * a family index outside [-1, nfamilies).  Host only. */
int32_t bx_family_grad(const double *dk_element, const int32_t *family, int32_t count,
                       int32_t nfamilies, double *dk_family);

/* Forward pass for differentiation: tracks the beam through the whole
 * lattice (all kicks, from a fresh state: no box, kick counter 0; space
 * charge as lattice->space_charge says), like bx_track but re-binning the
 * particles (when beam->id is given) before the first kick and at every
 * checkpoint, keeping each re-binning's particle map for the reverse pass,
 * and records in the context: the initial bunch, a checkpoint
 * (state and device tracking state) every `checkpoint_interval` kicks, the box
 * of every kick and every Green's function spectrum built.  box_replay (host,
 * may be NULL): 12 doubles per kick {lo[3], hi[3], h[3], 1/h[3]} as returned by
 * bx_grad_boxes; the box of each kick is then taken from it instead of the
 * box rule.  The beam arrays hold the final bunch afterwards.  Device memory
 * of the recording: about (ceil(K/C) + C + 3) * 48 + 4 * ceil(K/C) bytes per
 * particle plus C * 32 * n^3 + (K + 1) * 8 * (n+1)^3 bytes (K kicks, C = checkpoint_interval,
 * n = n_grid); allocated on the first call for a given size.  Asynchronous
 * except the allocation; BX_BAD_ARG for an empty beam or lattice. */
int32_t bx_grad_forward(bx_ctx *ctx, bx_beam *beam, const bx_lattice *lattice,
                        int32_t checkpoint_interval, const double *box_replay, void *stream);

/* Reverse pass after bx_grad_forward on the same beam (its final bunch):
 * weights (host, 4) as for L above.  dk_out (host, lattice count, may be
 * NULL) receives dL/dk per element (0 for non-quadrupoles, summed over the
 * element's slices); S_out (host, 36, may be NULL) receives
 * S[i*6 + j] = sum_p dL/dz0_i * z0_j; zbar0 (six device arrays of n, may be
 * NULL) receives dL/dz0 in the beam's particle order.  Recomputes each
 * checkpoint segment from its checkpoint, then runs the reverse kernels of
 * its kicks in reverse order.  Synchronous (waits for the stream); the
 * recording is consumed.  Results are bitwise reproducible. */
int32_t bx_grad_backward(bx_ctx *ctx, const bx_beam *beam, const double weights[4],
                         double *dk_out, double *S_out, double *const zbar0[6], void *stream);

/* Boxes of the last bx_grad_forward: up to `cap` kicks of 12 doubles
 * {lo[3], hi[3], h[3], 1/h[3]} into out (host); *count = kicks.  Synchronous. */
int32_t bx_grad_boxes(bx_ctx *ctx, double *out, int64_t cap, int64_t *count);

/* ---- Batches of independent tracking problems --------------------------
 * No counterpart in the paper: many lattice variants (e.g. a scan of
 * quadrupole strengths) or bunches of uneven particle counts and grid sizes
 * tracked at once.  Each problem is one context (its own grid size and
 * scratch), one beam and one lattice; bx_batch_launch runs every problem's
 * whole lattice, each exactly as bx_reset + bx_track(ctx, beam, lattice, 0,
 * -1) would (same kernels, same results bit for bit), as ONE CUDA graph
 * launch: the graph holds one independent branch per problem, a state reset
 * and the first half map followed by a device-side WHILE loop over that
 * problem's kick (the box-rule kernel of each kick decides whether another
 * kick follows and which optional parts run).  The problems' kernels
 * interleave on the GPU. */

/* Build the batch graph for `count` problems (ctxs[i], beams[i], lattices[i];
 * contexts distinct; the beams' arrays and ids must stay allocated and at the
 * same addresses while the batch exists).  Uploads each problem's map table
 * into its context, sizes its re-binning scratch, captures and instantiates
 * the graph.  Synchronous on `stream`.  Errors via bx_batch_last_error(NULL). */
int32_t bx_batch_create(bx_batch **out, int32_t count, bx_ctx *const *ctxs,
                        bx_beam *const *beams, const bx_lattice *const *lattices, void *stream);

/* One graph launch: every problem of the batch tracks its whole lattice from
 * its beam's current coordinates (fresh box and Green's function).
 * Asynchronous on `stream`; device errors surface through bx_sync of each
 * problem's context. */
int32_t bx_batch_launch(bx_batch *batch, void *stream);

/* Free the batch's graph (the contexts and beams are the caller's). */
int32_t bx_batch_destroy(bx_batch *batch);

/* Text of the last batch error (or of bx_batch_create when batch is NULL). */
const char *bx_batch_last_error(const bx_batch *batch);

/* ---- Tuning --------------------------------------------------------------
 * Re-binning interval, bin edge and cell order as in bx_options (takes effect
 * at the next call; BX_BAD_ARG for invalid values). */
int32_t bx_set_binning(bx_ctx *ctx, int32_t rebin_interval, int32_t bin_edge,
                       int32_t cell_order);

/* Autotuner of the binning (the bin and deposit layout; no result depends on
 * it): tracks `kicks` kicks of the lattice from kick 0 (from a fresh state)
 * once per candidate (never re-bin; and every 8, 16, 32 or 64 kicks, those
 * not longer than the timed kicks, with each valid bin edge among 4, 8, 16,
 * in bin order and in cell order), timing each with CUDA events, and keeps
 * the fastest (bx_set_binning).  The beam's coordinates and ids are restored
 * afterwards and the context is reset (bx_reset), so results do not depend on
 * the tuning.  chosen (host, 3): the chosen rebin_interval, bin_edge and
 * cell_order; ms (host, may be NULL): the time of candidate i for
 * i < min(cap, *count), candidates in the order above; *count: number of
 * candidates.  Needs the beam's id array.  Synchronous; uses 7 n doubles of
 * device scratch for the saved coordinates and ids while it runs. */
int32_t bx_autotune_binning(bx_ctx *ctx, bx_beam *beam, const bx_lattice *lattice,
                            int32_t kicks, int32_t chosen[3], double *ms, int32_t cap,
                            int32_t *count, void *stream);

/* ---- Particle-sharded tracking (one bunch over several processes) -------
 * ImpactX runs one simulation over many nodes when it is started with MPI
 * (paper: section ImpactX and the comments of Listing 1), with ABLASTR's
 * charge deposition and Poisson solve as the routines that cross ranks.
 * Here each process (rank) holds a share of the bunch's particles in its own
 * context and beam, and the ranks advance the same kicks in lockstep.  Per
 * kick, bx_track calls the caller's allreduce twice on the box inputs and
 * twice on the charge: MIN over the three order-preserving integer keys of the
 * rest-frame minima, MAX over those of the maxima, then SUM over the two
 * integer charge accumulators (n^3 values each, the hi and lo parts of the
 * 51-bit fixed-point CIC weights).  Every rank then applies the same box rule
 * to the same global extent, solves the same Poisson problem redundantly and
 * kicks its own particles.  The accumulators are exact integers, so the sum
 * does not depend on how the bunch is split: the kicked coordinates are
 * bitwise those of one process tracking the whole bunch. */
#define BX_OP_SUM 0
#define BX_OP_MIN 1
#define BX_OP_MAX 2

/* Combine `count` int64 values at DEVICE address buf over all ranks, in
 * place (every rank passes the same count and op, in the same order).  The
 * result must be in buf for work enqueued on `stream` after the callback
 * returns: enqueue a stream-ordered collective on `stream` (e.g. NCCL), or
 * synchronize `stream`, reduce through host memory and copy back before
 * returning.  Return 0 on success; anything else aborts the bx_track call with
 * BX_COLLECTIVE. */
typedef int32_t (*bx_allreduce_fn)(int64_t *buf, int64_t count, int32_t op, void *stream,
                                   void *user);

/* allreduce: the callback; user: passed to it; n_total: particles of the
 * whole bunch over all ranks (the macroparticle charge is
 * charge_sign * bunch_charge_C / n_total; every rank gives the whole bunch's
 * charge in its bx_beam).  A rank may hold no particles. */
typedef struct {
    bx_allreduce_fn allreduce;
    void *user;
    int64_t n_total;
} bx_shard;

/* Make the context's bx_track calls one rank of a sharded run (shard = NULL
 * ends it).  While it is set, bx_track launches each kick's kernels one by
 * one with the callbacks between them (no CUDA graphs: a collective need not
 * be capturable), and a beam with more than n_total particles is refused;
 * bx_track_diagnostics, bx_grad_forward, bx_autotune_binning and batches
 * refuse a sharded context (BX_BAD_ARG).  bx_deposit, bx_solve, bx_gather_kick
 * and bx_moments stay local to the rank. */
int32_t bx_set_shard(bx_ctx *ctx, const bx_shard *shard);

/* Wait for the stream and return the device status word (then clear it). */
int32_t bx_sync(bx_ctx *ctx, void *stream);

/* Text of the last error of this context (or of bx_create when ctx is NULL). */
const char *bx_last_error(const bx_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* BEAMTRACK_H */
