/*
 * pic_gb300.h -- C ABI of the GB300 (sm_103a) engine for the self-consistent
 * particle-in-cell / Monte Carlo collision cycle of a capacitive RF argon
 * discharge and the test-particle transport of sputtered Al atoms, after
 * Trieschmann, Schmidt & Mussenbrock, "Particle-in-Cell/Test-Particle
 * Simulations of Technological Plasmas" (arXiv:1607.04069).
 *
 * Conventions
 *   - Every function returns PIC_OK (0) or a negative PIC_ERR_* code;
 *     pic_strerror() names it and pic_last_error() gives the detail of the
 *     last failure on the calling thread.
 *   - "host" pointers are ordinary CPU memory owned by the caller; "device"
 *     pointers are CUDA global memory on the context's device, owned by the
 *     caller.  The context owns everything else it allocates.
 *   - Work is enqueued on the CUDA stream given to pic_create (a
 *     cudaStream_t passed as void*, NULL = legacy default stream) and runs
 *     asynchronously; functions that return host data synchronise that
 *     stream first.  A context must not be used by two threads at once.
 *   - Positions: with pos_precision 32 a position is the unsigned 32-bit
 *     fixed-point fraction of the gap, x = pos L / 2^32 (pos 0 marks a
 *     removed slot); with pos_precision 64 it is a double in cell units,
 *     xi = x / dx (negative marks a removed slot).  Test particles always
 *     use the 32-bit form.  Velocities are float32 (m/s), ids uint64.
 *   - Species: 0 = electrons, 1 = Ar+, 2 = sputtered Al test particles.
 */
#ifndef PIC_GB300_H
#define PIC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_OK 0
#define PIC_ERR_INVALID_ARG (-1)     /* a pointer, size or value is out of range          */
#define PIC_ERR_UNSTABLE_PARAMS (-2) /* strict mode: dx >= lambda_D or w_p dt >= 1       */
#define PIC_ERR_OUT_OF_MEMORY (-3)   /* device allocation failed                           */
#define PIC_ERR_CAPACITY (-4)        /* a birth or launch did not fit the slot capacity    */
#define PIC_ERR_NUMERICS (-5)        /* an electron exceeded the null-collision energy cap */
#define PIC_ERR_CUDA (-7)            /* a CUDA call failed (detail in pic_last_error)      */
#define PIC_ERR_NO_DEVICE (-8)       /* no CUDA device is visible                          */
#define PIC_ERR_TIMEOUT (-9)         /* pic_server_wait: the request had not finished;     */
                                     /* pic_sync: a kernel's bounded wait for a bulk copy  */
                                     /* gave up (the step's results are not valid)         */

enum pic_species { PIC_ELECTRON = 0, PIC_ION = 1, PIC_ATOM = 2 };

/* Discharge description.  SI units unless marked.  The discharge is the 1D
 * two-electrode setup of Sec. "Simulation Scenario": gap L, the left
 * electrode driven by the source V_rf(t), the right one grounded, argon at
 * constant pressure and temperature.  The source is V0 sin(2 pi f t) or
 * the paper's two-harmonic V0 [cos(2 pi f t + rf_phase) + cos(4 pi f t)],
 * and drives the electrode directly or through a series blocking capacitor
 * (surface-charge boundary condition, Sec. "EM Field Solver and External
 * Lumped Circuits"). */
typedef struct pic_params {
    double gap_m, pressure_pa, gas_temp_k, rf_freq_hz, rf_volt_v;
    double weight;          /* physical particles per superparticle per m^2 (Sec. "Kinetic
                               Particle Simulation": w = q_k / Q_k)                        */
    double dt;              /* PIC time step, s                                            */
    double te0_ev, ti0_ev;  /* temperatures of the initial uniform Maxwellian loading, eV  */
    double tp_dt;           /* test-particle time step used by tp_step(), s                */
    double sigma_tp;        /* Al-Ar hard-sphere cross section, m^2                        */
    int64_t n_e0, n_i0;     /* initial superparticles per charged species                  */
    int64_t cap_e, cap_i, cap_tp; /* slot capacity per species (0: 5/4 of the initial count
                                     plus 65536)                                          */
    uint64_t seed;          /* key of the Philox4x32-10 random stream                      */
    int32_t n_cells;        /* N cells (N+1 nodes); a power of two, 4..4096                */
    int32_t pos_precision;  /* 32 or 64, see "Positions" above                             */
    int32_t sputter_enable; /* Ar+ impacts launch Al test particles                        */
    int32_t tp_every;       /* coupled TP sub-cycle: one TP step of tp_every*dt after every
                               tp_every PIC steps (0 = none)                              */
    int32_t diag_every;     /* sampling stride of fluxes, EEDF and TP moments (0 = never)  */
    int32_t sort_every_e, sort_every_i, sort_every_tp; /* compaction periods (0 = never)   */
    int32_t ctas_per_sm;    /* CTAs per SM of the per-step launch (0 = occupancy limit)    */
    int32_t strict;         /* reject parameters violating dx < lambda_D or w_p dt < 1
                               (Sec. "Limitations and Constraints")                        */
    int32_t waveform;       /* 0: V0 sin(2 pi f t); 1: V0 [cos(2 pi f t + rf_phase) + cos(4 pi f t)] */
    int32_t circuit;        /* 0: the source sets the electrode potential; 1: the source drives
                               the electrode through the blocking capacitor c_block: per unit
                               area the capacitor holds q, the electrode carries q plus the
                               charge the particles brought to it (Gauss: eps0 E_0), and
                               phi_0 = V_rf - q / c_block                                 */
    double rf_phase;        /* waveform 1: phase of the fundamental, rad                    */
    double c_block;         /* circuit 1: capacitance per unit electrode area, F/m^2, >= 0
                               (0: floating electrode; INFINITY: same as circuit 0)        */
    int32_t tp_model;       /* Al-Ar collisions of the test particles (Sec. "Binary
                               Interactions"): 0 hard spheres of cross section sigma_tp;
                               1 VHS, sigma = pi b_max^2 with b_max(g) of Eq.
                               maximumimpactparameter, isotropic scattering; 2 M1, the same
                               law with d_ref sqrt(4/3) and chi = pi (1 - b / b_max)     */
    int32_t tp_mode;        /* collisions of tp_step (Sec. "Test Particle Method", Eq.
                               collisionprobability1 with a sampled Ar partner): 0 candidate
                               steps at a majorant probability, geometric gaps kept per atom,
                               thinned to the same per-step law; 1 the test drawn every step   */
    double tp_dref;         /* models 1, 2: VHS reference diameter of the Al-Ar pair, m (see
                               pic_vhs_dref)                                               */
    double tp_omega;        /* models 1, 2: viscosity index, 0.5 .. 1                      */
    double tp_tref;         /* models 1, 2: reference temperature, K                       */
    int64_t id_offset;      /* the initial loading holds particles id_offset .. id_offset +
                               n_e0 - 1 (and n_i0 - 1) of a larger loading (ids tag | k): one
                               rank's share when a discharge's particles are split over
                               ranks (see pic_exchange_slot); 0 for a whole discharge       */
} pic_params;

/* VHS reference diameter of a species from its viscosity mu_ref (Pa s) at
 * t_ref (K), viscosity index omega and molecular mass (kg), Eq.
 * referencediameter; for an unlike pair the paper averages the diameters and
 * the indices of the two species. */
double pic_vhs_dref(double mu_ref, double t_ref, double omega, double mass_kg);

/* Mono-energetic Ar+ source for tp_launch: n atoms leave the left electrode
 * with Sigmund-Thompson energies cut off at Lambda*e_ion_ev and cosine
 * angles (Sec. "Wall Interactions" of the test-particle method). */
typedef struct tp_source {
    int64_t n;
    double e_ion_ev;
    int64_t first_id;       /* the atoms get ids tag | (first_id + k), k < n; a negative value
                               continues after the atoms this context launched before.  A
                               source split over ranks gives each rank its own id range, and
                               the union is the one-rank source atom for atom            */
} tp_source;

typedef struct pic_ctx pic_ctx; /* opaque */

/* Fill *p with the 25 mm / 128-cell / 100 V / 3 Pa discharge. */
int pic_params_default(pic_params* p);

/* Create a discharge: validate p, allocate its state on the current CUDA
 * device, load n_e0 / n_i0 superparticles uniformly with Maxwellian
 * velocities (Sec. "Kinetic Particle Simulation": initial loading) and
 * solve the field of that state (Sec. "EM Field Solver").  `stream` is a
 * cudaStream_t or NULL.  On success *out owns the context. */
int pic_create(const pic_params* p, void* stream, pic_ctx** out);

/* Device bytes pic_create would allocate for p (capacities left at 0 take
 * their defaults); nothing is allocated.  For admission by memory budget. */
int pic_state_bytes(const pic_params* p, int64_t* bytes);

/* Release everything the context owns (waits for its stream). */
void pic_destroy(pic_ctx* ctx);

/* Advance n_steps PIC/MCC cycles (Sec. "Particle-In-Cell Scheme", Fig. 4:
 * field interpolation, leapfrog push (Eqs. pushinr, pushinv), wall
 * absorption with sputtered-atom launch, null-collision MCC (Sec. "Particle
 * Collisions"), linear charge assignment into exact int64 fixed point, and
 * the Poisson solve with the RF boundary value).  Periodic compaction and
 * coupled TP steps follow sort_every_* and tp_every.  Asynchronous: returns
 * the launch status; device-side conditions surface in pic_sync. */
int pic_step(pic_ctx* ctx, int64_t n_steps);

/* Wait for the context's stream; returns PIC_ERR_CAPACITY or
 * PIC_ERR_NUMERICS if the device recorded either since the last call. */
int pic_sync(pic_ctx* ctx);

/* One discharge whose superparticles are split over several contexts (one
 * per rank, each created with its id_offset and share of n_e0 / n_i0).  The
 * field solve of Sec. "EM Field Solver" needs the charge of all particles,
 * which is the sum of the ranks' exact int64 deposits (Sec. "Charge
 * Assignment"); every other part of the cycle is per particle, with random
 * words keyed by the particle's id, so the split run equals the whole one.
 * After pic_create and after every pic_step(ctx, 1), before the next step,
 * the caller sums this device block over the ranks in place (an int64 sum
 * all-reduce, e.g. NCCL on the context's stream): *dev receives the
 * context-owned device int64[*n_words] of the current step -- the electron
 * and ion deposits and their flux moments, padded with zeros.  The blocks
 * rotate over three buffers, one per step, so ask for the pointer after
 * every step (each stays valid for the context's life).  Time averages of
 * the charge, potential and fluxes are then those of the whole discharge on
 * every rank; histograms, counters and test particles stay per rank and add
 * up.  PIC_ERR_INVALID_ARG with circuit 1 (the series capacitor needs the
 * whole wall charge each step). */
int pic_exchange_slot(pic_ctx* ctx, int64_t** dev, int64_t* n_words);

/* Test of the bounded waits of the TP step (Sec. "Test Particle Method";
 * tp_step): with enable != 0, from the next TP step on, warp 0 of the first
 * CTA issues none of its bulk copies into shared memory, so its first wait
 * on a tile's barrier runs out (after 4096 polls instead of 2^22) with no
 * copy in flight.  The kernel sets its timeout bit, that warp's atoms do
 * not move, the launch completes, and the next pic_sync returns
 * PIC_ERR_TIMEOUT; the context stays usable.  enable = 0 restores the
 * normal step.  Waits for the stream first.  Intended for tests only. */
int pic_test_wait_timeout(pic_ctx* ctx, int enable);

/* Diagnostics (Sec. "Simulation Results", Figs. 5-9), written to host memory:
 *  0 PHI      time-averaged potential, V, N+1 nodes
 *  1 NE 2 NI  time-averaged densities, m^-3, N+1 nodes
 *  3 GAMMA_E 4 GAMMA_I  time-averaged particle fluxes, m^-2 s^-1
 *  5 VE 6 VI  mean velocities Gamma/n, m/s
 *  7 EEDF     electron energies in the central 10% of the gap, 256 x 0.25 eV
 *  8 IEDF_L 9 IEDF_R  Ar+ impact energies, 512 bins over [0, 2 V0]
 * 10 IEADF_L 11 IEADF_R  Ar+ impact energy x angle, 128 x 90 (energy-major)
 * 12 SPUTTER_E_L 13 SPUTTER_E_R  Al deposition energies, 600 x 0.5 eV
 * 14 SPUTTER_ANG_L 15 SPUTTER_ANG_R  Al deposition angles, 90 x 1 deg
 * 16 TP_DENS  time-averaged Al density, m^-3;  17 TP_V  Al mean v_x, m/s
 * 18 E        instantaneous field, V/m;  19 PHI_NOW  instantaneous potential
 * 20 TPF_TIME  event-driven TP flight (tp_flight): residence time summed over
 *              the atoms, s, per cell (N values; Sec. "Limitations and
 *              Constraints": time-weighted densities)
 * 21 TPF_VX    its mean v_x per cell (signed path / residence time), m/s
 * Histograms are raw counts.  Writes min(cap, size) values, *n_written = size. */
enum pic_diag_kind {
    PIC_DIAG_PHI = 0, PIC_DIAG_NE, PIC_DIAG_NI, PIC_DIAG_GAMMA_E, PIC_DIAG_GAMMA_I, PIC_DIAG_VE,
    PIC_DIAG_VI, PIC_DIAG_EEDF, PIC_DIAG_IEDF_L, PIC_DIAG_IEDF_R, PIC_DIAG_IEADF_L,
    PIC_DIAG_IEADF_R, PIC_DIAG_SPUTTER_E_L, PIC_DIAG_SPUTTER_E_R, PIC_DIAG_SPUTTER_ANG_L,
    PIC_DIAG_SPUTTER_ANG_R, PIC_DIAG_TP_DENS, PIC_DIAG_TP_V, PIC_DIAG_E, PIC_DIAG_PHI_NOW,
    PIC_DIAG_TPF_TIME, PIC_DIAG_TPF_VX, PIC_DIAG_COUNT
};
int pic_diag(pic_ctx* ctx, int kind, double* host_out, int64_t cap, int64_t* n_written);

/* The checks of the paper's two modelling assumptions (Sec. "Hypotheses
 * validation") from the time averages so far, into host_out[6]:
 *   [0], [1]  dE/E_max of the Ar+ energy distribution at x = 0 and x = L:
 *             full width at half maximum around the fullest bin over that
 *             bin's centre energy (mono-energetic impact, assumption A)
 *   [2], [3]  rms impact angle at x = 0 and x = L, degrees (normal impact)
 *   [4]       max over the nodes of n_Ar+ / n_Ar (assumption B)
 *   [5]       max over the nodes of n_Al / n_Ar (grid-based TP density)
 * A histogram without counts gives 0. */
int pic_hypotheses(pic_ctx* ctx, double* host_out);

/* Restart all time averages and histograms (Sec. "Kinetic Particle
 * Simulation": averaging once a (periodic) steady state is reached). */
int pic_reset_averages(pic_ctx* ctx);

/* Event counters, host int64[cap]: n_e, n_i, n_tp (slots in use), step,
 * tp_step, impacts e L/R, Ar+ L/R, ionisations, sputtered L/R, Al deposited
 * L/R, numerics, elastic, excitation, CX, isotropic, TP collisions,
 * capacity.  Synchronises.  *n_written = number of counters (23). */
int pic_counters(pic_ctx* ctx, int64_t* host_out, int64_t cap, int64_t* n_written);

/* Copy the alive particles of one species to host buffers of length cap
 * (any may be NULL): xi = x/dx (double, cell units), vx, vy, vz, id.
 * *n_out = number alive (may exceed cap; then only cap are written). */
int pic_get_species(pic_ctx* ctx, int species, int64_t cap, double* xi, float* vx, float* vy,
                    float* vz, uint64_t* id, int64_t* n_out);

/* Replace the particles of one species by n host-side particles.  pos is in
 * the storage form of the species (uint32 or double, see "Positions").  The
 * field is re-solved for the new state unless keep_field is nonzero. */
int pic_set_species(pic_ctx* ctx, int species, int64_t n, const void* pos, const float* vx,
                    const float* vy, const float* vz, const uint64_t* id, int keep_field);

/* Instantaneous field state, host double/int64 arrays of N+1 (any may be
 * NULL): E (V/m), phi (V), and the last deposit q_e, q_i in units of 2^-32
 * superparticles per node. */
int pic_get_field(pic_ctx* ctx, double* E, double* phi, int64_t* q_e, int64_t* q_i);

/* Overwrite the nodal field used by the next step's interpolation. */
int pic_set_field(pic_ctx* ctx, const double* E);

/* Launch sputtered atoms from a mono-energetic source (see tp_source). */
int tp_launch(pic_ctx* ctx, const tp_source* src);

/* Advance the test particles n_steps of tp_dt (Sec. "Test Particle Method":
 * free flight, sticking at the walls, hard-sphere collisions with a thermal
 * Ar partner).  If n_alive is not NULL the stream is synchronised and the
 * number of atoms still in flight is returned. */
int tp_step(pic_ctx* ctx, int64_t n_steps, int64_t* n_alive);

/* Event-driven (gridless) flight of the test particles (Sec. "Kinetic
 * Particle Simulation": free flight between collisions; Sec. "Limitations
 * and Constraints": time-weighted densities): each live atom flies straight
 * for tau = -ln(R) / nu(v) to its next collision or to an electrode, nu(v) =
 * n sigma_tp <|v - w|> over the Maxwellian gas; at an electrode it sticks
 * (Al deposition histograms and counters, as tp_step); otherwise it collides
 * as a hard sphere with a partner drawn from the gas weighted by |v - w|.
 * Each atom goes through at most max_events events in this call (launches of
 * up to 32 events each; the call returns early once no atom is alive).
 * Residence time and path are added per cell (PIC_DIAG_TPF_TIME, _VX).
 * Synchronises the stream; *n_alive (may be NULL) receives the atoms still
 * in flight. */
int tp_flight(pic_ctx* ctx, int64_t max_events, int64_t* n_alive);

/* Tabulate the e-Ar cross section of process q (0 elastic, 1 excitation,
 * 2 ionisation) from n host points (energy in eV, increasing; sigma in m^2,
 * >= 0), as LXcat-style data are given (Sec. "Particle Collisions": cross
 * sections from look-up tables): linear between the points, constant beyond
 * the ends; n = 0 restores the analytic form.  The thresholds of the
 * kinematics (11.5 and 15.8 eV) stay.  nu_max follows from the tables'
 * largest values, and every electron's next null-collision candidate is
 * drawn afresh from the current step.  Synchronises the stream. */
int pic_set_cross_section(pic_ctx* ctx, int process, int64_t n, const double* energy_ev, const double* sigma_m2);

/* Compact one species now (drop removed slots, counting sort by cell). */
int pic_compact(pic_ctx* ctx, int species);

/* CUDA-event timing of the per-step kernel launches on the context's stream.
 * pic_timing(ctx, 1) starts recording; pic_kernel_time returns the summed
 * device time (ms) and launch count of kind 0 = PIC step kernel,
 * 1 = TP step kernel, 2 = compaction, since timing was (re)enabled. */
int pic_timing(pic_ctx* ctx, int enable);
int pic_kernel_time(pic_ctx* ctx, int kind, double* ms, int64_t* launches);

/* Phase trace of the per-step launch (tracing aid): pic_trace(ctx, 1)
 * allocates a device buffer into which every CTA of each subsequent step
 * launch writes 16 words -- globaltimer stamps (ns) at start, after loading
 * the deposit, after the field solve, at the end of the prologue, after the
 * particle stream, after the queued events, after the histogram flush and at
 * exit; its species; its event count (low 32 bits) and touched node range
 * (high 32 bits); stamps after the launch set-up and after issuing the
 * deposit copies; the longest single event (ns << 8 | event kind); its
 * ionisations; the longest tile-flush thread (ns); one unused word.
 * pic_trace_read copies the words of the last launch (grid x 16) to host
 * memory; *n_written = grid x 16.  pic_trace(ctx, 0) frees the buffer. */
int pic_trace(pic_ctx* ctx, int enable);
int pic_trace_read(pic_ctx* ctx, uint64_t* host_out, int64_t cap, int64_t* n_written);

/* Derived quantities of the discharge, host double[8]: n_gas, dx,
 * nu_max_e, nu_max_i, P_max_e, P_max_i, eps_max, Lambda. */
int pic_derived(pic_ctx* ctx, double* host_out8);

/* ---- stateless hot-path operations on caller device buffers ---- */

/* Linear (cloud-in-cell) charge assignment (Sec. "Charge Assignment"):
 * adds 2^32 - floor(f 2^32) to node j and floor(f 2^32) to node j+1 for each
 * of the n particles at device positions pos (uint32 fixed point when
 * pos_precision = 32, double cell units when 64), j = floor(xi), f = xi - j.
 * Removed slots are skipped.  q: device int64[n_cells+1], accumulated into
 * (not cleared).  Exact and independent of particle order. */
int pic_op_deposit(const void* pos, int pos_precision, int64_t n, int32_t n_cells, int64_t* q,
                   void* stream);

/* Field solve (Sec. "EM Field Solver"): from device int64 node counts q_i,
 * q_e (units of 2^-32 superparticles of weight w), solve
 * (phi[m+1] - 2 phi[m] + phi[m-1]) / dx^2 = -rho[m]/eps0 with phi[0] =
 * v_left, phi[N] = 0, and E = -dphi/dx (central inside, half-cell Gauss on
 * the electrodes).  phi, E: device double[n_cells+1]. */
int pic_op_poisson(const int64_t* q_i, const int64_t* q_e, int32_t n_cells, double dx, double weight,
                   double v_left, double* phi, double* E, void* stream);

/* Counting sort by cell of a caller-owned particle set, allocating no device
 * memory (the paper has no counterpart: this is the compaction of
 * pic_compact for callers that cannot call cudaMalloc or any allocating
 * routine, e.g. inside a host framework that owns all device memory).
 *   pos_precision  32 (pos: uint32 fixed point) or 64 (pos: double cell units);
 *   n              slots in the input, 0 <= n < 2^32;
 *   n_cells        power of two in [4, 4096]; larger values are rejected with
 *                  PIC_ERR_INVALID_ARG because the scratch is a fixed 32 KiB
 *                  __device__ array inside the library (4096 counts + 4096
 *                  offsets of 32 bits);
 *   pos..id        device input arrays of n slots (removed slots -- pos 0,
 *                  or negative xi -- and positions outside [0, n_cells) are
 *                  dropped);
 *   *_out          device output arrays with room for n slots, written in
 *                  cell order (order within a cell is unspecified); they must
 *                  not overlap the inputs;
 *   n_out          device int64 receiving the number kept, or NULL;
 *   stream         cudaStream_t as void*, NULL = legacy default stream.
 * The work runs asynchronously on `stream`.  Every call looks up the scratch
 * array's address with the current device (cudaGetSymbolAddress), so a
 * device reset between calls is harmless; the first call on a device also
 * loads the library's kernels there, so make it before any stream capture.
 * All calls share the one scratch
 * array: each call clears the counts it uses, and calls whose work may
 * overlap on the GPU (other streams, other host threads) race on it, so the
 * caller must order them. */
int pic_op_sort_noalloc(int pos_precision, int64_t n, int32_t n_cells, const void* pos, const float* vx,
                        const float* vy, const float* vz, const uint64_t* id, void* pos_out, float* vx_out,
                        float* vy_out, float* vz_out, uint64_t* id_out, int64_t* n_out, void* stream);

/* ------------------------------------------------------------ batches
 * Several independent discharges (for instance a scan over pressure or RF
 * voltage) stepped together: one step launch per time step covers every
 * member, each member owning a contiguous range of that launch's CTAs.  The
 * paper has no counterpart; each member runs the same PIC/MCC cycle as
 * pic_step (Sec. "Particle-In-Cell Scheme", Fig. 4) and its results are bit
 * for bit those of the same discharge stepped alone.
 *
 * Members use 32-bit positions, one dt and one diag_every, a whole number
 * of steps per RF period (1 / (f dt) integral, at most 2^24), and no coupled
 * test-particle steps (tp_every 0).  The RF phase of step l is taken at
 * l mod period in both forms.  A member joins (pic_batch_add) only while every
 * current member stands at a multiple of diag_every steps, so that all of
 * them sample on the same steps.  Each member keeps 2 or more CTAs,
 * ceil((n_e0 + n_i0) / particles_per_cta) of them; by default (0) the
 * division is automatic: two waves of resident CTAs over all members'
 * particles, clamped to [2048, 16384] particles per CTA. */
typedef struct pic_batch pic_batch; /* opaque */

/* Create an empty batch whose work goes to `stream` (cudaStream_t or NULL). */
int pic_batch_create(void* stream, pic_batch** out);

/* Create a member from p (as pic_create does, on the batch's stream) and
 * return its slot index in *slot (the lowest free one).  The member starts
 * at step 0. */
int pic_batch_add(pic_batch* b, const pic_params* p, int* slot);

/* Destroy the member in `slot` (waits for the batch's stream); the slot
 * becomes free and the other members keep their slots and state. */
int pic_batch_remove(pic_batch* b, int slot);

/* The member's context, for pic_diag / pic_counters / pic_get_species /
 * pic_sync.  Owned by the batch: do not pic_destroy it, and do not
 * pic_step it while it belongs to the batch. */
int pic_batch_ctx(pic_batch* b, int slot, pic_ctx** out);

/* Particles per CTA when the launch is divided among members (>= 1024, or
 * 0 for the automatic division). */
int pic_batch_set_target(pic_batch* b, int64_t particles_per_cta);

/* How the launch runs those CTA slots.  particles_per_chunk > 0 (default
 * 131072): a grid of resident CTAs (a few per SM) takes chunks of
 * consecutive slots of one member from a work counter, paying the member's
 * deposit copy and field solve once per chunk instead of once per slot; a
 * chunk holds at most 1/(2R) of all slots (R resident CTAs), so a small
 * batch still spreads over every SM, and the last fifth of each member's
 * slots form one-slot chunks at the end, so the launch ends on short work.
 * 0: one CTA per slot, scheduled by the hardware.  The members' results are
 * the same either way. */
int pic_batch_set_chunk(pic_batch* b, int64_t particles_per_chunk);

/* Advance every member n_steps steps (one launch per step plus each
 * member's due compactions).  Asynchronous, as pic_step. */
int pic_batch_step(pic_batch* b, int64_t n_steps);

/* enable != 0: from the next pic_batch_step on, each run of diag_every
 * steps that starts on a multiple of diag_every and contains no member's
 * compaction before its last step is replayed from a CUDA graph of those
 * launches (captured once, again after the membership changes).  Results
 * are unchanged. */
int pic_batch_graphs(pic_batch* b, int enable);

/* Waits for the batch's stream, writes to *ms / *steps (host, may be NULL)
 * the device time of the step launches and graph replays recorded since the
 * last call and the steps they covered (compactions excluded), clears both,
 * and turns recording on (enable != 0) or off. */
int pic_batch_timing(pic_batch* b, int enable, double* ms, int64_t* steps);

/* Choose the particles-per-CTA division of the launch: for each of the
 * n_cand candidates (host array; NULL or n_cand 0: 8192 ... 262144 by
 * powers of two) run one untimed step and steps_each timed steps, then keep
 * the candidate with the least time per step (written to *best, may be
 * NULL).  These are real steps of every member: the division changes no
 * result, only the time. */
int pic_batch_autotune(pic_batch* b, const int64_t* candidates, int n_cand, int64_t steps_each, int64_t* best);

/* pic_sync on every member; returns the first error. */
int pic_batch_sync(pic_batch* b);

/* Destroy every member and the batch. */
void pic_batch_destroy(pic_batch* b);

/* ------------------------------------------------------------ serving
 * A request loop that runs submitted discharges to periodic steady state.
 * The paper has no counterpart; each discharge runs the PIC/MCC cycle of
 * pic_step, and steady state is the criterion of its Sec. "Simulation
 * Results": the cycle-averaged quantities no longer change from one RF
 * period to the next.
 *
 * One worker thread (started by pic_server_create on the current device,
 * with its own stream) admits queued requests in arrival order while the
 * sum of their state sizes (pic_state_bytes) stays within the budget, keeps
 * every admitted discharge resident, and steps them all together -- one
 * pic_batch, or one pic_step call per discharge when batched is 0 -- in
 * chunks of 1/chunks_per_period of an RF period (admission happens between
 * chunks).  At the end of each window of window_periods RF periods it reads
 * the discharge's window-averaged n_e and n_i; once at least min_periods
 * periods have run and the relative change of both from the window before
 * is below tol, the request completes with state CONVERGED (or MAX_PERIODS
 * when max_periods > 0 periods have run), its last window-averaged n_e, n_i
 * and phi are kept on the host and its device state is released.  Every
 * request needs a whole number of steps per RF period (else FAILED).  The
 * first request admitted while nothing runs sets the chunk; a later request
 * joins only if its period is a multiple of the chunk and the chunk a
 * multiple of its diag_every, and otherwise waits at the head of the queue
 * until the running discharges have finished (the chunk is then set anew).
 * Batched, a request also follows the pic_batch rules (32-bit positions,
 * one dt and diag_every; else FAILED).  A state larger than the whole
 * budget completes as REJECTED.  The change is that of
 * the inventory, the spatial integral of the density (criterion
 * PIC_STEADY_INVENTORY, the default: in steady state generation and losses
 * balance, Sec. "Simulation Results"), or of the profile in L2 over the
 * nodes (PIC_STEADY_PROFILE, which the statistical noise of small
 * discharges can keep above tol).  All functions are
 * thread-safe.  Times are seconds on the server's monotonic clock
 * (pic_server_clock), zero at creation. */
typedef struct pic_server pic_server; /* opaque */

typedef struct pic_server_opts {
    int64_t hbm_budget_bytes;  /* device bytes the resident discharges may hold; 0: 80% of free memory */
    int32_t min_periods;       /* RF periods before the steady-state test (>= 2)             */
    int32_t max_periods;       /* a request ends after this many periods (0: no limit)       */
    double tol;                /* steady state: relative L2 change of n_e and n_i below tol  */
    int32_t batched;           /* 1: one batch launch per step; 0: a plain loop of pic_step   */
    int32_t graphs;            /* batched: replay sampling periods from CUDA graphs          */
    int32_t chunks_per_period; /* admission / check granularity (default 10)                  */
    int32_t criterion;         /* PIC_STEADY_INVENTORY (default) or PIC_STEADY_PROFILE        */
    int32_t window_periods;    /* RF periods per averaging window (>= 1, default 1)           */
    int32_t pad;
} pic_server_opts;

enum pic_steady_criterion { PIC_STEADY_INVENTORY = 0, PIC_STEADY_PROFILE = 1 };

enum pic_request_state {
    PIC_REQ_QUEUED = 0, PIC_REQ_RUNNING, PIC_REQ_CONVERGED, PIC_REQ_MAX_PERIODS, PIC_REQ_REJECTED,
    PIC_REQ_FAILED
};

typedef struct pic_request_info {
    int64_t id;
    int32_t state;             /* pic_request_state                                          */
    int32_t periods;           /* RF periods completed                                       */
    double t_arrival, t_admit, t_done;   /* server clock (s); -1 until reached               */
    double change;             /* last period-to-period relative change (-1 before the 2nd)  */
    int64_t bytes;             /* device bytes of the discharge's state                      */
    int64_t particles;         /* initial superparticles, e- + Ar+                            */
} pic_request_info;

typedef struct pic_server_stats {
    int64_t queued, running, done;       /* requests in each phase                          */
    int64_t bytes_used, budget;          /* device bytes held by admitted requests; budget   */
    int64_t chunks, steps;               /* step chunks the worker ran, and their steps      */
    double particle_steps;               /* sum over chunks of initial particles x steps     */
    double busy_s;                       /* worker time spent in the chunks                  */
} pic_server_stats;

/* Defaults: budget 0 (80% of free), min_periods 2, max_periods 0, tol 0.01,
 * batched 1, graphs 1, chunks_per_period 10, criterion inventory,
 * window_periods 1. */
int pic_server_opts_default(pic_server_opts* o);
/* opts may be NULL (defaults). */
int pic_server_create(const pic_server_opts* opts, pic_server** out);
int pic_server_clock(pic_server* s, double* t);
/* Queue a request; t_arrival (server clock, <= now; negative: now) is the
 * time latency is measured from.  *id receives the request id. */
int pic_server_submit(pic_server* s, const pic_params* p, double t_arrival, int64_t* id);
/* Current state of a request (host struct, written by the call). */
int pic_server_info(pic_server* s, int64_t id, pic_request_info* info);
/* Block until the request has finished (timeout_s < 0: no limit); returns
 * PIC_ERR_TIMEOUT if it has not within timeout_s.  info may be NULL. */
int pic_server_wait(pic_server* s, int64_t id, double timeout_s, pic_request_info* info);
/* Why a request FAILED or was REJECTED (NUL-terminated, at most cap bytes). */
int pic_server_error(pic_server* s, int64_t id, char* out, int64_t cap);
/* The last window-averaged profile of a request: what 0 = n_e, 1 = n_i
 * (m^-3), 2 = phi (V), n_cells + 1 node values into host `out` (cap
 * doubles; *n receives the count, 0 before the first window ends). */
int pic_server_result(pic_server* s, int64_t id, int what, double* out, int64_t cap, int64_t* n);
/* Drop a finished request's record. */
int pic_server_forget(pic_server* s, int64_t id);
/* Counters of the server (host struct); PIC_ERR_CUDA if the worker stopped
 * on a device error (every running request then FAILED). */
int pic_server_status(pic_server* s, pic_server_stats* out);
/* Stop the worker (running requests are abandoned) and free everything.  No
 * other pic_server_* call on s may be running or start while it runs. */
void pic_server_destroy(pic_server* s);

const char* pic_strerror(int code);
const char* pic_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PIC_GB300_H */
