/*
 * lb.h -- C ABI of the GB300 (sm_103a) thermal pseudopotential D3Q19 lattice Boltzmann step.
 *
 * Method: Biferale, Perlekar, Sbragaglia, Toschi, "Convection in multiphase flows using
 * Lattice Boltzmann methods" (arXiv:1111.0905), "Algorithm" paragraph, Eqs. (6)-(9), with
 * the boundary conditions of the Fig. 1 caption and of the text around Eq. (4), and the
 * heat-flux diagnostic of Eqs. (4)-(5).
 *
 * Lattice (the paper names D3Q19 but fixes no ordering): l = 0 rest; 1..6 = (+-1,0,0),
 * (0,+-1,0), (0,0,+-1); 7..10 = (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0); 11..14 = (1,0,1),
 * (-1,0,-1),(1,0,-1),(-1,0,1); 15..18 = (0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1). Opposite pairs
 * (1,2),(3,4),...,(17,18). Weights 1/3, 1/18 (axis), 1/36 (diagonal).
 *
 * Grid: nx*ny*nz nodes, node index idx = x + nx*(y + ny*z) (x fastest). Periodic in x and
 * y; halfway no-slip walls at z = -1/2 (temperature T_d) and z = nz - 1/2 (T_u).
 * Field arrays are float64, nx*ny*nz long, in node-index order.
 * Population arrays are float64 [19][nx*ny*nz] (structure of arrays, l slowest).
 *
 * Ownership: the caller owns every array it passes; the context owns all device state
 * (two ping-pong population lattices f and g, diagnostics scratch). Device pointers must
 * be valid on the context's device and ordered on its stream.
 *
 * Errors: every int-returning call returns LB_OK (0) or a negative LB_E* code. Nothing is
 * printed, nothing exits, no device trap is used. lb_last_error() gives the context's last
 * message (for LB_ECUDA the CUDA error string).
 *
 * Threading: a context is used by one host thread at a time. All calls are ordered on the
 * context's CUDA stream; calls that return host data synchronise that stream.
 */
#ifndef THERMAL_LBM_LB_H
#define THERMAL_LBM_LB_H

#ifdef __cplusplus
extern "C" {
#endif

#define LB_OK 0
#define LB_EINVAL (-1)    /* invalid argument or parameter (tau <= 1/2, size, null pointer) */
#define LB_ENOMEM (-2)    /* device or host allocation failed */
#define LB_ECUDA (-3)     /* a CUDA call or kernel launch failed; see lb_last_error */
#define LB_ENONPHYS (-4)  /* health check found rho <= 0, T <= 0 or a NaN */
#define LB_EIO (-5)       /* checkpoint file could not be written/read or failed its checksum */
#define LB_EUNSUP (-6)    /* operation not supported for this precision/configuration */

/* Storage/compute precision of the populations. */
typedef enum {
  LB_FP64 = 0,     /* float64 storage and compute */
  LB_FP32 = 1,     /* float32 storage and compute */
  LB_BF16_DEV = 2, /* bfloat16 storage of the deviations below, float32 compute */
  LB_FP16_DEV = 3, /* float16 storage of the deviations below, float32 compute */
  LB_FP16_LOC = 4  /* float16 storage against local references (below), float32 compute */
} lb_precision;
/* LB_FP64 .. LB_FP16_DEV store deviations from the reference equilibria, f_l - f^eq_l(rho0, 0, T0)
 * and g_l - g^eq_l(rho0, T0, 0), and form moments and equilibria from them. LB_FP16_LOC stores,
 * per population, its deviation minus the rest equilibrium of the node that wrote it (its density
 * and temperature at that step, per lattice direction class, kept in FP16 in two extra slots per
 * lattice and node: 21 instead of 19 stored values), so that FP16 rounds the non-equilibrium and
 * velocity parts only. Measured against the float64 step (max over the field relative to its
 * scale): float32 stays within 1e-6 on rho and T over 2000 single-phase steps and 5e-5 over 5000
 * boiling steps of the 256^3 cell; float16 deviations within 2e-3 over 2000 single-phase steps but
 * not over long boiling runs (4e-2 after 5000 steps: the phase pattern drifts); bfloat16 deviations
 * only over a few tens of steps (within 2e-3 after 50 steps of a 32^3 cell, 3.8e-3 after 100 steps
 * of the 512^3 boiling cell); float16 against local references within 2e-3 over both horizons
 * (2.3e-4 after 5000 boiling steps of the 256^3 cell). */

/* Scheme variants for comparison with the paper's scheme (variant 0 of each; the paper defines
 * neither alternative). Forcing: LB_FORCE_SHIFT, the paper's equilibrium velocity
 * u' = (j + tau_nu F)/rho; LB_FORCE_GUO, f^eq at the physical velocity u = (j + F/2)/rho plus
 * (1 - 1/(2 tau_nu)) w_l [3 (c_l - u).F + 9 (c_l.u)(c_l.F)] (Guo, Zheng, Shi, PRE 65, 046308).
 * Pseudopotential: LB_PSI_EXP, psi = exp(-1/rho) of the "Algorithm" paragraph; LB_PSI_VDW,
 * psi = rho sqrt(2 (a - b T_v/(1 - b rho))/(-G)) (G < 0), whose bulk pressure
 * rho T + (G/2) psi^2 carries the non-ideal van der Waals pressure at temperature T_v. */
#define LB_FORCE_SHIFT 0
#define LB_FORCE_GUO 1
#define LB_PSI_EXP 0
#define LB_PSI_VDW 1

typedef struct {
  int nx, ny, nz;         /* grid; each >= 1, 19*nx*ny*nz < 2^32 */
  double tau_nu;          /* f relaxation time, Eq. (6); > 1/2 */
  double tau_kappa;       /* g relaxation time, Eq. (7); > 1/2 */
  double G;               /* pseudopotential coupling of Eq. (9); bulk P = rho T + (G/2) e^{-2/rho} */
  double kappa;           /* thermal conductivity, Eqs. (2)-(3); > 0 */
  double c_v;             /* specific heat at constant volume, Eq. (3); > 0 (1 = default) */
  double g_z;             /* signed gravity along z, Eq. (1) (negative = downward) */
  double T_d, T_u;        /* bottom / top wall temperatures */
  double rho0, T0;        /* reference state of the deviation storage; <= 0: mean of the init fields */
  int precision;          /* lb_precision */
  int nu_every;           /* > 0: accumulate Nu_mean every nu_every steps into the time average */
  int check_every;        /* > 0: lb_step checks rho > 0, T > 0, no NaN every check_every steps */
  int tile_y;             /* launch shape: CTA tile is 32 x tile_y (4, 8 or 16; 16 not with FP64;
                             0 = default: 8) */
  int z_chunk;            /* launch shape: planes per CTA (0 = choose from the grid size) */
  int forcing;            /* LB_FORCE_SHIFT (0, the paper) or LB_FORCE_GUO */
  int psi_kind;           /* LB_PSI_EXP (0, the paper) or LB_PSI_VDW */
  double vdw_a, vdw_b;    /* LB_PSI_VDW: attraction a > 0 and excluded volume b > 0 */
  double vdw_T;           /* LB_PSI_VDW: temperature T_v > 0 of the non-ideal pressure; b T_v < a
                             (1 - b rho) must hold for every density the run reaches */
} lb_params;

typedef struct lb_ctx lb_ctx;  /* opaque */

/* lb_init -- allocate a context and set the initial state f = f^eq(rho, 0, T), g = g^eq(rho, T, 0)
 * ("Algorithm" paragraph: equilibria of Eqs. (6)-(7) at rest).
 * rho_init, T_init: float64 fields (node-index order), host memory if init_on_device == 0,
 * device memory otherwise; copied, not retained. cuda_stream: a cudaStream_t (NULL = the
 * legacy default stream) on the current device; every later call is ordered on it.
 * On success *out is the new context. Errors: LB_EINVAL (parameters, an unknown variant, a
 * van der Waals psi that is not real at some initial density, rho <= 0 or T <= 0 or
 * non-finite input), LB_ENOMEM, LB_ECUDA. On error *out is NULL and nothing is leaked. */
int lb_init(const lb_params* params, const double* rho_init, const double* T_init,
            int init_on_device, void* cuda_stream, lb_ctx** out);

/* lb_step -- advance nsteps time steps of Eqs. (6)-(7): per step one fused launch that pull-
 * streams f and g (periodic x/y, bounce-back walls), takes the moments of Eq. (8), the force of
 * Eq. (9) with psi = exp(-1/rho) plus gravity rho g_z z (psi_kind selects the variant), the shifted
 * velocity u' = (j + tau_nu F)/rho (forcing selects the variant),
 * the physical velocity u = (j + F/2)/rho and its divergence, and collides f (temperature in
 * f^eq) and g (with the counter term -rho T div u / c_v). Asynchronous on the context's stream
 * unless nu_every/check_every ask for host-visible checks. nsteps >= 0.
 * Errors: LB_EINVAL, LB_ECUDA (launch), LB_ENONPHYS (health check failed, e.g. a density beyond
 * the range where the van der Waals psi is real; the state is kept). */
int lb_step(lb_ctx* ctx, long long nsteps);

/* lb_moments -- macroscopic fields of the current state (Eq. (8)): rho, the physical velocity
 * u = (j + F/2)/rho and T = (sum_l g_l)/rho. Each output is float64 [nx*ny*nz]; host memory if
 * on_device == 0 (the call synchronises), device memory otherwise. Any output may be NULL.
 * Errors: LB_EINVAL, LB_ENOMEM, LB_ECUDA. */
int lb_moments(lb_ctx* ctx, double* rho, double* ux, double* uy, double* uz, double* T,
               int on_device);

/* lb_nusselt -- layer heat flux of Eq. (4) as a Nusselt number,
 * Nu(z) = <rho U u_z - kappa dT/dz>_{x,y} / (kappa (T_d - T_u)/nz), U = c_v T + (G/4) e^{-2/rho}
 * (Eq. (2); for the van der Waals psi U = c_v T - T_v ln(1 - b rho) - a rho), dT/dz by central
 * differences with wall ghosts 2 T_wall - T. Host outputs: *nu_mean = mean over z; nu_z (may be
 * NULL) = nz values; *nu_time_avg (may be NULL) = mean of the Nu_mean samples accumulated by
 * lb_step with nu_every > 0 (NaN if none). Warp sums in the compute precision, FP64 across warps,
 * tiles and planes in a fixed order (deterministic); synchronises. Errors: LB_EINVAL, LB_ECUDA. */
int lb_nusselt(lb_ctx* ctx, double* nu_mean, double* nu_z, double* nu_time_avg);

/* lb_adjoint_step -- advance nsteps steps from the current state (as lb_step) and return the
 * time-averaged Nusselt number J = (1/nsteps) sum_{n=1..nsteps} Nu_mean(state n) (Eq. (4)) with its
 * exact discrete gradient by reverse mode: dJ/dT_d, dJ/dT_u, dJ/dG and, if dJ_dT0 is not NULL,
 * dJ/dT0 (host float64 [nx*ny*nz]) with respect to the temperature field passed to lb_init (then
 * the context must be at step 0). The paper defines no adjoint; the reverse pass transposes the
 * operations of lb_step (streaming and wall rules, f and g collisions with the counter term, the
 * velocities and divergence, the force of Eq. (9) with psi = exp(-1/rho), the moments of Eq. (8))
 * in FP64 around the forward states of the context's precision, which are recomputed segment by
 * segment from checkpoints taken every checkpoint_every steps (with FP64 storage the recomputing
 * step writes the fields the reverse sweep needs; the last segment's come from the forward
 * sweep). J is accumulated in the reverse sweep from the identity Nu_mean = 1 + sum_x rho U u_z /
 * (kappa (T_d - T_u) nx ny) (the conduction term telescopes). Output pointers may be NULL.
 * Device memory: nsteps/checkpoint_every + 1 population checkpoints, checkpoint_every + 1 sets of
 * 20 float64 fields, 3 float64 states and 15 float64 fields, allocated and freed by the call.
 * checkpoint_every = 0 takes the longest segment whose buffers fit in 85 % of the device's free
 * memory: all nsteps states' fields when they fit (with FP64 storage nothing is then recomputed),
 * else the largest length that fits.
 * Synchronises. Errors: LB_EINVAL (nsteps < 1, checkpoint_every < 0, T_d == T_u, dJ_dT0 requested
 * after lb_step), LB_EUNSUP (a scheme variant: the reverse pass transposes the paper's scheme
 * only), LB_ENOMEM (also: no segment length fits), LB_ECUDA. */
int lb_adjoint_step(lb_ctx* ctx, long long nsteps, int checkpoint_every, double* J,
                    double* dJ_dTd, double* dJ_dTu, double* dJ_dG, double* dJ_dT0);

/* lb_populations -- the current pre-collision state (f_l, g_l) as float64 [19][nx*ny*nz] each
 * (Eqs. (6)-(7): populations after streaming). Host memory if on_device == 0. Either pointer
 * may be NULL. Errors: LB_EINVAL, LB_ENOMEM, LB_ECUDA. */
int lb_populations(lb_ctx* ctx, double* f, double* g, int on_device);

/* lb_set_populations -- replace the current state by a given pre-collision state (f_l, g_l), float64
 * [19][nx*ny*nz] each in the layout of lb_populations (Eqs. (6)-(7): populations after streaming,
 * before the collision of the next step); host memory if on_device == 0 (the call synchronises),
 * device memory otherwise. The values are stored in the context's precision as given (no
 * validation: the health check of lb_step reports a non-physical state). The step count and the
 * accumulated Nu samples are kept; a sample due for the replaced state is dropped. Afterwards
 * lb_adjoint_step gives no dJ/dT0 (the state is no longer lb_init's equilibrium). The paper has no
 * counterpart (it restarts from stored populations, e.g. for comparisons at an evolved state).
 * Errors: LB_EINVAL (null argument), LB_ENOMEM, LB_ECUDA. */
int lb_set_populations(lb_ctx* ctx, const double* f, const double* g, int on_device);

/* lb_diagnostics -- health and conservation of the current state, on the host:
 * out[0] = min rho, out[1] = min T, out[2] = count of non-finite rho/T/u, out[3] = total mass
 * sum rho, out[4] = total sum rho T. FP64 reductions. Errors: LB_EINVAL, LB_ECUDA. */
int lb_diagnostics(lb_ctx* ctx, double out[5]);

/* lb_profiles -- per-plane means of the current state (the T(z) profile and its asymmetry, Fig. 2
 * top inset, and the P div(u) term of the integral constraint of Eq. (5)): rho_z[z] = <rho>_{x,y},
 * T_z[z] = <T>_{x,y}, PdivU_z[z] = <P div(u)>_{x,y} with P = rho T + (G/2) e^{-2/rho} and the
 * divergence of the physical velocity by central differences (u_z -> -u_z across the walls).
 * Host outputs of nz values; any may be NULL. FP64 sums in a fixed order. Synchronises.
 * Errors: LB_EINVAL, LB_ENOMEM, LB_ECUDA. */
int lb_profiles(lb_ctx* ctx, double* rho_z, double* T_z, double* PdivU_z);

/* lb_histogram_T_rho -- joint histogram of (T, rho) of the nodes in planes [z_lo, z_hi) (the T-rho
 * scatter of Fig. 2 top, per region): counts[iT * nrho + irho] (host, uint64, nT * nrho <= 12288),
 * bin = floor((v - lo) / (hi - lo) * n) for lo <= v < hi; values outside are not counted.
 * Synchronises. Errors: LB_EINVAL (ranges), LB_ENOMEM, LB_ECUDA. */
int lb_histogram_T_rho(lb_ctx* ctx, int z_lo, int z_hi, int nT, double T_lo, double T_hi, int nrho,
                       double rho_lo, double rho_hi, unsigned long long* counts);

/* lb_structure_functions -- horizontal structure functions of the vertical velocity and of the
 * temperature over the planes [z_lo, z_hi) (Eq. (10), Fig. 3): for r = 1..rmax (rmax < nx, ny),
 * S2_q[r-1] = <dq^2>, S4_q[r-1] = <dq^4> with dq = q(x + r e) - q(x) averaged over e = e_x, e_y
 * (periodic) and all nodes of the planes; the flatness is S4 / S2^2. Host outputs of rmax values,
 * any may be NULL. FP64 sums in a fixed order. Synchronises. Errors: LB_EINVAL, LB_ENOMEM, LB_ECUDA. */
int lb_structure_functions(lb_ctx* ctx, int rmax, int z_lo, int z_hi, double* S2_uz, double* S4_uz,
                           double* S2_T, double* S4_T);

/* lb_heat_flux_pdf -- statistics of the local convective heat flux q = rho U u_z (U = c_v T plus the
 * non-ideal internal energy; the bulk term of Nu in Eq. (4), whose pdf in the bulk is the inset of
 * Fig. 2) over the planes [z_lo, z_hi): counts (host uint64 [nbins], 1 <= nbins <= 12288) of the
 * nodes with q_lo <= q < q_hi, bin = floor((q - q_lo)/(q_hi - q_lo) nbins), and stats (host
 * double [3]) = number of nodes, mean and variance of q over every node of the planes (FP64,
 * fixed-order sums, variance from the deviations from the mean). Either output may be NULL.
 * Synchronises. Errors: LB_EINVAL, LB_ENOMEM, LB_ECUDA. */
int lb_heat_flux_pdf(lb_ctx* ctx, int z_lo, int z_hi, int nbins, double q_lo, double q_hi,
                     unsigned long long* counts, double* stats);

/* lb_save / lb_load -- checkpoint of (parameters, step count, populations in their storage
 * precision) to a raw binary file with a header and a 64-bit FNV-1a checksum of the payload.
 * lb_load requires a context created with the same grid, precision and physics parameters
 * (tau_nu, tau_kappa, G, kappa, c_v, g_z, T_d, T_u, forcing, psi_kind and, for the van der Waals
 * psi, its a, b, T_v; the launch shape and sampling periods may differ) and replaces its state,
 * step count, Nu time average and deviation reference rho0, T0.
 * Errors: LB_EINVAL, LB_EIO (open/write/read failure, bad magic, grid/precision/parameter
 * mismatch, checksum), LB_ECUDA. */
int lb_save(lb_ctx* ctx, const char* path);
int lb_load(lb_ctx* ctx, const char* path);

/* lb_step_count -- number of steps taken since lb_init (or restored by lb_load); -1 if ctx is NULL. */
long long lb_step_count(const lb_ctx* ctx);

/* lb_launch_info -- how the context's step kernel is launched (launch metadata for performance
 * reports; the paper has no counterpart). Host output of 6 ints: out[0], out[1] = grid (column
 * tiles, z chunks), out[2] = threads per CTA, out[3] = dynamic shared memory bytes per CTA,
 * out[4] = CTAs resident per SM as the CUDA occupancy calculator reports it, out[5] = registers
 * per thread. Errors: LB_EINVAL (NULL argument), LB_ECUDA. */
int lb_launch_info(lb_ctx* ctx, int* out);

/* lb_free -- release the context and its device memory (synchronises its stream). NULL is a no-op. */
void lb_free(lb_ctx* ctx);

/* lb_strerror -- static description of an LB_E* code. */
const char* lb_strerror(int code);

/* lb_last_error -- the context's last error message ("" if none); a static message if ctx is NULL. */
const char* lb_last_error(const lb_ctx* ctx);

/* lb_nusselt_fields_noalloc -- Nu(z) of lb_nusselt computed from caller-owned device fields, for
 * callers that cannot allocate device memory (an application whose own pool allocator owns all
 * device memory, or a latency-critical loop that cannot take cudaMalloc's implicit
 * synchronisation). The paper has no counterpart; it is a variant of the Nusselt reduction of
 * the diagnostics path. It allocates nothing: its per-plane partial sums live in a fixed
 * file-scope device array of 2 * LB_NOALLOC_MAX_NZ doubles (128 KB) that every GPU loading the
 * library keeps until the process exits.
 * Inputs (device, float64, node-index order, nx*ny*nz each): rho, uz (physical velocity, z),
 * T, e.g. written by lb_moments with on_device = 1. Output (device, float64): nu_out[0..nz-1] =
 * Nu(z), nu_out[nz] = mean over z. Parameters as in lb_params. The internal energy is that of
 * the paper's pseudopotential only, U = c_v T + (G/4) e^{-2/rho}: for fields of a context with
 * psi_kind = LB_PSI_VDW this call does not give lb_nusselt's Nu (use lb_nusselt there).
 * Enqueued on cuda_stream (NULL = legacy default stream) of the current device; nothing is
 * synchronised. Launch failures are read from the launch calls themselves; an error left pending
 * in the CUDA runtime by the caller's earlier work is neither cleared nor reported.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) and
 * keeps it; make that first call before any stream capture. The kept address does not survive
 * cudaDeviceReset of that device: do not call this entry point after such a reset. Every call
 * shares the array: calls that overlap on the GPU (other streams, other threads) race and must be
 * ordered by the caller. Each call writes every partial it reads, so no state carries over between
 * calls.
 * Errors: LB_EINVAL (null pointer, nx/ny/nz < 1, nz > LB_NOALLOC_MAX_NZ, kappa <= 0, c_v <= 0,
 * T_d == T_u), LB_ECUDA (symbol lookup or launch failed). */
#define LB_NOALLOC_MAX_NZ 8192
int lb_nusselt_fields_noalloc(const double* rho, const double* uz, const double* T,
                              int nx, int ny, int nz, double kappa, double G, double c_v,
                              double T_d, double T_u, double* nu_out, void* cuda_stream);

/* lb_stream_bound -- a measurement aid, not a physical step: the memory access pattern of one
 * time step (streaming of Eqs. (6)-(7): 19 f and 19 g pulled from the neighbours x - c_l, 19 + 19
 * values written) with none of its arithmetic. For every node and direction l, f_out[l][node] =
 * f_in[l][source] and g_out[l][node] = g_in[l][source], source = node - c_l, periodic in x and y,
 * z clamped into [0, nz) (the step bounces back at the walls instead; the clamp keeps the same
 * locality). Lattices [19][nz][ny][nx] in the library's direction order (0 rest, 1..6 axis +-x,
 * +-y, +-z, 7..10 xy, 11..14 xz, 15..18 yz diagonals), elements of elem_bytes = 4 (float) or 2
 * (any 16-bit type: bits are copied), device memory, caller-owned; the outputs must not overlap
 * the inputs. Its bandwidth at the fused step's residency is the bound of the step's access
 * pattern there.
 * ctas_per_sm: 0 = one node per thread (256-thread CTAs covering the cell); k >= 1 = a single
 * resident wave of SMs * k CTAs of 256 threads striding over the nodes (8k warps per SM).
 * max_ctas_per_sm (may be NULL) receives the kernel's occupancy limit; a larger ctas_per_sm is
 * refused. Enqueued on cuda_stream (NULL = legacy default stream) of the current device; nothing
 * is synchronised.
 * Errors: LB_EINVAL (null lattice pointer, nx/ny/nz < 1, 19 nx ny nz >= 2^32, elem_bytes not 2 or
 * 4, ctas_per_sm < 0 or above the occupancy limit), LB_ECUDA (device query or launch failed). */
int lb_stream_bound(int elem_bytes, const void* f_in, const void* g_in, void* f_out, void* g_out,
                    int nx, int ny, int nz, int ctas_per_sm, int* max_ctas_per_sm, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* THERMAL_LBM_LB_H */
