/*
 * pic_oracle.c -- plain, slow, FP64 CPU oracle of the 1d3v electrostatic
 * particle-in-cell / Monte Carlo collision (PIC/MCC) cycle and of the
 * test-particle (TP) transport of sputtered atoms described in
 * Trieschmann, Schmidt & Mussenbrock, "Particle-in-Cell/Test-Particle
 * Simulations of Technological Plasmas" (arXiv:1607.04069).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path calls this file:
 * it exists so that tests, the smoke check and the CPU-baseline leg of the
 * benchmark can check the CUDA path against an independent implementation.
 * It shares no code, header, table or constant with the CUDA path; both are
 * written from the same paper and the same readings of it.
 *
 * Style: every particle is processed in index order with plain loops; no
 * blocking, no fusion, no reordering beyond what the paper's cycle states
 * (Sec. "Particle-In-Cell Scheme", Fig. 4: charge assignment -> field solve
 * -> field interpolation -> push -> wall interaction -> collisions).
 *
 * Positions are kept in units of the cell size, xi = x / dx, so that the
 * linear-weighting rule (Sec. "Charge Assignment") is evaluated exactly for
 * positions that the GPU path stores as 32-bit fixed point.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), counter
 * (id_lo, id_hi, step, purpose), key (seed_lo, seed_hi).  The purpose codes
 * are listed below; they define which random word is used for what.
 *
 * Parity pins for every function here live in tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- physical constants (CODATA 2018 exact/recommended values) ---- */
#define O_QE 1.602176634e-19      /* elementary charge, C          */
#define O_ME 9.1093837015e-31     /* electron mass, kg             */
#define O_AMU 1.66053906660e-27   /* atomic mass unit, kg          */
#define O_KB 1.380649e-23         /* Boltzmann constant, J/K       */
#define O_EPS0 8.8541878128e-12   /* vacuum permittivity, F/m      */
#define O_PI 3.14159265358979323846
#define O_MAR (39.948 * O_AMU)    /* argon atom / ion mass         */
#define O_MAL (26.98 * O_AMU)     /* aluminium atom mass           */

/* ---- analytic cross sections and surface model (readings of the paper) ---- */
#define O_SIG_EL 1e-19            /* e-Ar elastic, m^2, constant          */
#define O_EXC_TH 11.5             /* e-Ar excitation threshold, eV        */
#define O_EXC_SIG 1e-20           /* excitation magnitude scale, m^2      */
#define O_ION_TH 15.8             /* e-Ar ionisation threshold, eV        */
#define O_LOTZ_A 4.5e-18          /* Lotz constant a, m^2 eV^2            */
#define O_LOTZ_Q 6.0              /* Lotz shell occupation q              */
#define O_ARP_SIG 5e-19           /* Ar+-Ar iso and CX: 5e-19 (1eV/eps)^.5 */
#define O_UB 3.4                  /* Al surface binding energy, eV        */
#define O_SP_TH 30.0              /* sputter threshold, eV                */
#define O_SP_MAXN 16              /* at most 16 sputter trials per impact */

/* ---- random-stream purposes (the third/fourth counter words) ---- */
enum {
    PUR_INIT = 1,        /* initial loading: step word 0 and 1          */
    PUR_COLL = 2,        /* per-step candidate test, process, direction */
    PUR_IONIZE = 3,      /* ionisation energy split, ejected direction  */
    PUR_NEWION = 4,      /* Maxwellian velocity of the newborn ion      */
    PUR_BIRTH_ID = 5,    /* ids of the ionisation children              */
    PUR_GAS = 6,         /* gas partner of an Ar+ collision             */
    PUR_GAP = 7,         /* steps to the next candidate, after one      */
    PUR_GAP0 = 8,        /* steps to the first candidate, on entry      */
    PUR_SP_TRIAL = 16,   /* +k/4: sputter trials                        */
    PUR_SP_EMIT = 32,    /* +k: energy/angle of the k-th sputtered atom */
    PUR_SP_ID = 48,      /* +k: id of the k-th sputtered atom           */
    PUR_TP_GAS = 64,     /* gas partner of a TP step                    */
    PUR_TP_COLL = 65,    /* TP collision test and scattering direction  */
    PUR_TP_LAUNCH = 66,  /* mono-energetic source launch                */
    PUR_TPF_FLIGHT = 70, /* event-driven TP: free-flight time of event e */
    PUR_TPF_SCATTER = 71,/* event-driven TP: scattering direction       */
    PUR_TPF_PARTNER = 72,/* +2t, +2t+1: partner proposal t of event e    */
    PUR_TPF_CAND = 200,  /* VHS/M1 flight: candidate partner (200, 201)  */
    PUR_TPF_GAMMA = 202, /* +t: gamma variate attempt t of a candidate   */
    PUR_TP_CAND = 256,   /* TP step candidate: partner proposal (256, 257) */
    PUR_TP_GAMMA = 258,  /* +t: gamma variate attempt t of that proposal  */
    PUR_TP_GAP = 290,    /* TP steps to the next candidate, after one     */
    PUR_TP_GAP0 = 291    /* TP steps to the first candidate              */
};
#define TPF_GAMMA_TRIES 32
#define TPF_TRIES 64     /* partner proposals per collision (each accepted w.p. >= 1/2) */

/* species and id tags (top two bits of the 64-bit id) */
#define SP_E 0
#define SP_I 1
#define SP_TP 2
static const uint64_t TAG[3] = {0ull, 1ull << 62, 2ull << 62};
#define ID_MASK ((1ull << 62) - 1)

/* histogram shapes */
#define NB_IEDF 512    /* ion energy, [0, 2 V0] eV            */
#define NB_IEADF_E 128 /* IEADF energy bins, [0, 2 V0] eV     */
#define NB_ANG 90      /* 1-degree angle bins, [0, 90) deg     */
#define NB_EEDF 256    /* 0.25 eV bins, [0, 64) eV             */
#define NB_SPE 600     /* 0.5 eV bins, [0, 300) eV              */

/* counters exported by orc_counters() */
enum {
    C_NE, C_NI, C_NTP, C_IMP_E_L, C_IMP_E_R, C_IMP_I_L, C_IMP_I_R, C_IONIZ,
    C_SPUT_L, C_SPUT_R, C_TPDEP_L, C_TPDEP_R, C_NUMERICS, C_ELASTIC, C_EXCIT,
    C_CX, C_ISO, C_TPCOLL, C_CAPACITY, C_NCOUNT
};

/* Discharge parameters (SI units unless marked). */
typedef struct {
    double L, p, Tg, f, V0;       /* gap, pressure, gas T, RF frequency, amplitude */
    double w, dt;                 /* superparticle weight (1/m^2), time step       */
    double te0, ti0;              /* initial temperatures, eV                      */
    double tp_dt, sigma_tp;       /* TP time step for orc_tp_step, hard-sphere xs  */
    uint64_t seed;
    int32_t ncell;                /* N cells, N+1 nodes                            */
    int32_t sputter;              /* ion impacts launch sputtered atoms            */
    int32_t tp_every;             /* coupled TP sub-cycle (0: no coupled TP)       */
    int32_t diag_every;           /* flux / EEDF sampling stride                   */
    int32_t waveform;             /* 0: V0 sin(wt); 1: V0 [cos(wt + phase) + cos 2wt] */
    int32_t circuit;              /* 0: the source sets phi[0]; 1: series capacitor  */
    double phase;                 /* waveform 1: phase of the fundamental, rad      */
    double cb;                    /* circuit 1: capacitance per electrode area, F/m^2 */
    double dref, omega, tref;     /* TP models 1, 2: VHS reference diameter (m), viscosity index,
                                     reference temperature (K) of the Al-Ar pair   */
    int32_t tp_model;             /* TP collisions: 0 hard sphere (sigma_tp), 1 VHS, 2 M1 */
    int32_t coll_mode;            /* null-collision candidates of e- and Ar+: 0 geometric gaps
                                     between candidates (orc_gap), 1 the paper's literal test,
                                     a fresh R <= P_c,tot every step                   */
    int32_t tp_mode;              /* TP step collisions: 0 candidates at a majorant rate with
                                     geometric gaps, thinned to the per-step law
                                     (orc_tp_step), 1 the literal test every step     */
    int32_t pad2;
} orc_params;

typedef struct {
    int64_t n, cap;
    double *xi, *vx, *vy, *vz;
    uint64_t *id;
    uint32_t *nev;                /* step of the next null-collision candidate */
    uint8_t *alive;
} orc_sp;

typedef struct {
    orc_params P;
    orc_sp sp[3];
    double *E, *phi;
    int64_t *q[2];
    uint32_t step, tp_step;
    /* derived quantities */
    double ngas, dx, nu_max_e, nu_max_i, p_max_e, p_max_i, eps_max;
    double lam[2];                /* nu_max dt of e- and Ar+                    */
    /* diagnostics */
    double *sum_q[2], *sum_phi, *sum_flux[2], *tp_dens, *tp_vx;
    double *tpf_time, *tpf_disp;  /* event-driven TP: residence time (s), signed path (m) per cell */
    double *xs_e[3], *xs_s[3];    /* tabulated e-Ar cross sections (eV, m^2), or NULL: analytic */
    int64_t xs_n[3];
    int64_t n_avg, n_flux, n_tp_samp, tp_launched;
    double tp_gap_dt;             /* TP dt the stored candidate gaps were drawn for     */
    int64_t *iedf[2], *ieadf[2], *eedf, *sp_e[2], *sp_ang[2];
    int64_t cnt[C_NCOUNT];
} orc_state;

/* ======================= Philox4x32-10 (Salmon et al. 2011) ============== */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(uint64_t seed, uint64_t id, uint32_t step, uint32_t purpose, uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox(ctr, key, out);
}

/* uniform in (0,1): the top 23 bits of a word plus one half, times 2^-23 */
static double u23(uint32_t w) { return ((double)(w >> 9) + 0.5) * 0x1p-23; }

/* Box-Muller (Sec. "Kinetic Particle Simulation": Maxwellian sampling) */
static void box_muller(uint32_t a, uint32_t b, double *n1, double *n2)
{
    double r = sqrt(-2.0 * log(u23(a)));
    double t = 2.0 * O_PI * u23(b);
    *n1 = r * cos(t);
    *n2 = r * sin(t);
}

/* uniform direction on the unit sphere: cos(theta) = 1 - 2R, phi = 2 pi R */
static void iso_dir(uint32_t a, uint32_t b, double d[3])
{
    double c = 1.0 - 2.0 * u23(a);
    double s = sqrt(fmax(0.0, 1.0 - c * c));
    double ph = 2.0 * O_PI * u23(b);
    d[0] = c; d[1] = s * cos(ph); d[2] = s * sin(ph);
}

static uint64_t child_id(uint32_t lo, uint32_t hi, int species)
{
    return ((((uint64_t)hi << 32) | lo) & ID_MASK) | TAG[species];
}

/* ======================= cross sections ================================== */
/* electron-argon, eps in eV, result in m^2 (Sec. "Particle Collisions") */
void orc_sigma_e(double eps, double out[3])
{
    out[0] = O_SIG_EL;
    out[1] = eps > O_EXC_TH ? O_EXC_SIG * (1.0 - O_EXC_TH / eps) : 0.0;
    out[2] = eps > O_ION_TH ? O_LOTZ_A * O_LOTZ_Q * log(eps / O_ION_TH) / (eps * O_ION_TH) : 0.0;
}

/* Tabulated cross section (Sec. "Particle Collisions": energy-dependent
 * cross sections from look-up tables): linear interpolation between the
 * points (E_i, sigma_i), E increasing, held constant beyond the first and
 * last points. */
double orc_xs_interp(const double *E, const double *sg, int64_t n, double eps)
{
    if (eps <= E[0]) return sg[0];
    if (eps >= E[n - 1]) return sg[n - 1];
    int64_t lo = 0, hi = n - 1;                  /* E[lo] <= eps < E[hi] */
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (E[mid] <= eps) lo = mid; else hi = mid;
    }
    return sg[lo] + (eps - E[lo]) / (E[hi] - E[lo]) * (sg[hi] - sg[lo]);
}

/* the three e-Ar cross sections at eps: tabulated where a table is set */
static void electron_sigma(const orc_state *S, double eps, double out[3])
{
    orc_sigma_e(eps, out);
    for (int p = 0; p < 3; p++)
        if (S->xs_n[p]) out[p] = orc_xs_interp(S->xs_e[p], S->xs_s[p], S->xs_n[p], eps);
}

/* Ar+-Ar isotropic and charge exchange (each channel), eps in eV */
double orc_sigma_i(double eps) { return O_ARP_SIG * sqrt(1.0 / eps); }

/* sputter yield of Al by Ar+ at normal incidence, E in eV */
double orc_yield(double E) { return E > O_SP_TH ? 0.1 * sqrt(E / O_SP_TH - 1.0) : 0.0; }

/* maximum fraction of energy passed in a binary Ar -> Al collision */
static double lambda_ar_al(void) { return 4.0 * O_MAR * O_MAL / ((O_MAR + O_MAL) * (O_MAR + O_MAL)); }

/* Sigmund-Thompson energy E/(E+Ub)^3 truncated at Emax and cosine angle
 * (Sec. "Wall Interactions" of the TPM): energy from the inverse of the
 * truncated CDF (E/(E+Ub))^2, polar angle theta = arccos(sqrt(R)), azimuth
 * 2 pi R.  dir = +1 launches into +x (left electrode), -1 into -x. */
void orc_emit(double uE, double uT, double uP, double Emax, double dir, double v[3])
{
    double Fmax = (Emax / (Emax + O_UB)) * (Emax / (Emax + O_UB));
    double s = sqrt(uE * Fmax);
    double Es = O_UB * s / (1.0 - s);
    double speed = sqrt(2.0 * Es * O_QE / O_MAL);
    double ct = sqrt(uT);
    double st = sqrt(fmax(0.0, 1.0 - uT));
    double ps = 2.0 * O_PI * uP;
    v[0] = dir * speed * ct;
    v[1] = speed * st * cos(ps);
    v[2] = speed * st * sin(ps);
}

/* ======================= charge assignment =============================== */
/* Linear (cloud-in-cell) weighting (Sec. "Charge Assignment"): a particle
 * at xi in cell j = floor(xi), f = xi - j, gives 2^32 - floor(f 2^32) to node
 * j and floor(f 2^32) to node j+1, so each particle deposits exactly 2^32.
 * Particles with xi < 0 are treated as removed. */
void orc_deposit(const double *xi, int64_t n, int32_t ncell, int64_t *q)
{
    for (int64_t k = 0; k < n; k++) {
        if (!(xi[k] >= 0.0)) continue;
        double j = floor(xi[k]);
        double f = xi[k] - j;
        int64_t wr = (int64_t)floor(f * 4294967296.0);
        int64_t wl = 4294967296LL - wr;
        int64_t m = (int64_t)j;
        if (m < 0 || m >= ncell) continue;
        q[m] += wl;
        q[m + 1] += wr;
    }
}

/* ======================= field solve ===================================== */
/* Poisson (Sec. "EM Field Solver"): (phi[m+1] - 2 phi[m] + phi[m-1])/dx^2 =
 * -rho[m]/eps0 on interior nodes, phi[0] = v_left, phi[N] = 0, solved with
 * the Thomas algorithm.  rho[m] = e w (q_i - q_e) / (2^32 V_m) with node
 * volume V_m = dx inside and dx/2 on the electrodes.  E[m] = -(phi[m+1] -
 * phi[m-1])/(2 dx) inside; on the electrodes Gauss's law over the half cell. */
void orc_poisson(int32_t N, double dx, double w, const int64_t *q_i, const int64_t *q_e,
                 double v_left, double *phi, double *E)
{
    double *rho = (double *)malloc(sizeof(double) * (N + 1));
    double *cp = (double *)malloc(sizeof(double) * (N + 1));
    double *dp = (double *)malloc(sizeof(double) * (N + 1));
    for (int m = 0; m <= N; m++) {
        double vol = (m == 0 || m == N) ? 0.5 * dx : dx;
        rho[m] = O_QE * w * (double)(q_i[m] - q_e[m]) / (4294967296.0 * vol);
    }
    phi[0] = v_left;
    phi[N] = 0.0;
    if (N >= 2) {
        /* rows m = 1..N-1: a = 1, b = -2, c = 1 */
        for (int m = 1; m <= N - 1; m++) {
            double d = -dx * dx * rho[m] / O_EPS0;
            if (m == 1) d -= phi[0];
            if (m == N - 1) d -= phi[N];
            if (m == 1) {
                cp[m] = 1.0 / -2.0;
                dp[m] = d / -2.0;
            } else {
                double den = -2.0 - cp[m - 1];
                cp[m] = 1.0 / den;
                dp[m] = (d - dp[m - 1]) / den;
            }
        }
        phi[N - 1] = dp[N - 1];
        for (int m = N - 2; m >= 1; m--) phi[m] = dp[m] - cp[m] * phi[m + 1];
    }
    for (int m = 1; m <= N - 1; m++) E[m] = -(phi[m + 1] - phi[m - 1]) / (2.0 * dx);
    E[0] = (phi[0] - phi[1]) / dx - rho[0] * dx / (2.0 * O_EPS0);
    E[N] = (phi[N - 1] - phi[N]) / dx + rho[N] * dx / (2.0 * O_EPS0);
    free(rho); free(cp); free(dp);
}

/* ======================= state =========================================== */
static void sp_alloc(orc_sp *s, int64_t cap)
{
    s->n = 0; s->cap = cap;
    s->xi = (double *)calloc(cap ? cap : 1, sizeof(double));
    s->vx = (double *)calloc(cap ? cap : 1, sizeof(double));
    s->vy = (double *)calloc(cap ? cap : 1, sizeof(double));
    s->vz = (double *)calloc(cap ? cap : 1, sizeof(double));
    s->id = (uint64_t *)calloc(cap ? cap : 1, sizeof(uint64_t));
    s->nev = (uint32_t *)calloc(cap ? cap : 1, sizeof(uint32_t));
    s->alive = (uint8_t *)calloc(cap ? cap : 1, 1);
}

static void sp_free(orc_sp *s)
{
    free(s->xi); free(s->vx); free(s->vy); free(s->vz); free(s->id); free(s->nev); free(s->alive);
}

static double mass_of(int s) { return s == SP_E ? O_ME : (s == SP_I ? O_MAR : O_MAL); }
static double charge_of(int s) { return s == SP_E ? -O_QE : (s == SP_I ? O_QE : 0.0); }

/* Null-collision candidates (Sec. "Particle Collisions"): every step a
 * particle is a candidate with the fixed probability P_c,tot = 1 -
 * exp(-nu_max dt), independently of the other steps.  Two equivalent
 * procedures are kept:
 *  - coll_mode 1, the paper's own: each step draws R = Philox(id, l, COLL)
 *    word 0 and the particle is a candidate iff R < P_c,tot;
 *  - coll_mode 0: the number of steps from one candidate to the next is
 *    geometric, P(gap = n) = exp(-nu_max dt (n-1)) (1 - exp(-nu_max dt)), and
 *    is drawn as the free flight time of Sec. "Kinetic Particle Simulation",
 *    tau = -tau_c ln R with tau_c = 1 / nu_max, counted in steps and rounded
 *    up: gap = 1 + floor(-ln R / (nu_max dt)).  Each particle keeps the step
 *    of its next candidate.
 * A candidate then uses the same words in both: Philox(id, l, COLL) words 1-3
 * for the process and the scattering direction. */
uint32_t orc_gap(double lam, uint32_t w)
{
    double x = -log(u23(w)) / lam;
    if (!(x < 2147483646.0)) return 2147483647u;
    return 1u + (uint32_t)floor(x);
}

/* step of the first candidate of a particle that is first pushed at step l0 */
static uint32_t entry_nev(const orc_state *S, int s, uint64_t id, uint32_t l0)
{
    if (s == SP_TP) return 0;
    uint32_t c[4];
    draw(S->P.seed, id, l0, PUR_GAP0, c);
    return l0 - 1u + orc_gap(S->lam[s], c[0]);
}

static int64_t append(orc_state *S, int s, double xi, double vx, double vy, double vz, uint64_t id,
                      uint32_t l0)
{
    orc_sp *p = &S->sp[s];
    if (p->n >= p->cap) { S->cnt[C_CAPACITY]++; return -1; }
    int64_t k = p->n++;
    p->xi[k] = xi; p->vx[k] = vx; p->vy[k] = vy; p->vz[k] = vz; p->id[k] = id; p->alive[k] = 1;
    p->nev[k] = entry_nev(S, s, id, l0);
    return k;
}

/* Source voltage at step l (Sec. "Simulation Scenario"): a sine of
 * amplitude V0, or the fundamental and its second harmonic,
 * V0 [cos(w t + phase) + cos(2 w t)], whose relative phase makes a
 * geometrically symmetric discharge electrically asymmetric. */
double orc_source_voltage(const orc_state *S, uint32_t l)
{
    double wt = 2.0 * O_PI * S->P.f * (double)l * S->P.dt;
    if (S->P.waveform == 1) return S->P.V0 * (cos(wt + S->P.phase) + cos(2.0 * wt));
    return S->P.V0 * sin(wt);
}

/* Electrode potential with the source in series with a blocking capacitor
 * (Sec. "Simulation Scenario", Sec. "EM Field Solver and External Lumped
 * Circuits": the surface charge couples plasma and circuit).  Per unit
 * electrode area the capacitor holds q; the left electrode carries sigma =
 * q + w, w the charge the particles have delivered to it (ions minus
 * electrons absorbed there since creation); Gauss's law over the half cell
 * ties sigma to the field at the electrode, sigma = eps0 E_0; and the loop
 * gives phi_0 = V - q/c.  E_0 is linear in phi_0: E_0 = E_0(charge, phi_0 =
 * 0) + phi_0 E_0(no charge, phi_0 = 1), both from the discrete Poisson
 * problem, so phi_0 = (c V - eps0 E_0(charge, 0) + w) / (c + eps0 E_0(no
 * charge, 1)).  An infinite c is the ideal source, phi_0 = V; c = 0 is a
 * floating electrode, sigma = w. */
static double circuit_potential(orc_state *S, double V)
{
    if (isinf(S->P.cb)) return V;
    int N = S->P.ncell;
    double *phi = (double *)malloc(sizeof(double) * (N + 1));
    double *E = (double *)malloc(sizeof(double) * (N + 1));
    int64_t *zero = (int64_t *)calloc(N + 1, sizeof(int64_t));
    orc_poisson(N, S->dx, S->P.w, S->q[SP_I], S->q[SP_E], 0.0, phi, E);
    double e_charge = E[0];
    orc_poisson(N, S->dx, S->P.w, zero, zero, 1.0, phi, E);
    double e_unit = E[0];
    free(phi); free(E); free(zero);
    double w = O_QE * S->P.w * (double)(S->cnt[C_IMP_I_L] - S->cnt[C_IMP_E_L]);
    return (S->P.cb * V - O_EPS0 * e_charge + w) / (S->P.cb + O_EPS0 * e_unit);
}

static double v_rf(orc_state *S, uint32_t l)
{
    double V = orc_source_voltage(S, l);
    return S->P.circuit ? circuit_potential(S, V) : V;
}

/* deposit both charged species and solve the field for time step l */
static void deposit_all(orc_state *S)
{
    int N = S->P.ncell;
    for (int s = 0; s < 2; s++) {
        memset(S->q[s], 0, sizeof(int64_t) * (N + 1));
        orc_sp *p = &S->sp[s];
        for (int64_t k = 0; k < p->n; k++) {
            if (!p->alive[k]) continue;
            orc_deposit(&p->xi[k], 1, N, S->q[s]);
        }
    }
}

static void solve_for_step(orc_state *S, uint32_t l)
{
    orc_poisson(S->P.ncell, S->dx, S->P.w, S->q[SP_I], S->q[SP_E], v_rf(S, l), S->phi, S->E);
}

static void field_for_step(orc_state *S, uint32_t l)
{
    deposit_all(S);
    solve_for_step(S, l);
}

/* derived quantities of the null-collision method (Sec. "Particle
 * Collisions"): nu_max is the maximum over energy of n sigma_sum(eps)
 * sqrt(2 eps / m_r).  Electrons: the sum of the closed-form maxima of the
 * three cross sections at the highest admitted energy eps_max = 2 V_peak + 100 eV
 * (V_peak = V0 for the sine, 2 V0 for the two-harmonic waveform).
 * Ar+: sigma(eps) g is constant, so nu_max is exact. */
static void derive(orc_state *S)
{
    orc_params *P = &S->P;
    S->ngas = P->p / (O_KB * P->Tg);
    S->dx = P->L / (double)P->ncell;
    S->eps_max = 2.0 * (P->waveform == 1 ? 2.0 * P->V0 : P->V0) + 100.0;   /* peak source voltage */
    double sig_max[3] = {O_SIG_EL, O_EXC_SIG, O_LOTZ_A * O_LOTZ_Q / (exp(1.0) * O_ION_TH * O_ION_TH)};
    for (int q = 0; q < 3; q++)                  /* a table: its largest value */
        if (S->xs_n[q]) {
            sig_max[q] = 0.0;
            for (int64_t i = 0; i < S->xs_n[q]; i++) sig_max[q] = fmax(sig_max[q], S->xs_s[q][i]);
        }
    double sig_sum_max = sig_max[0] + sig_max[1] + sig_max[2];
    S->nu_max_e = S->ngas * sig_sum_max * sqrt(2.0 * S->eps_max * O_QE / O_ME);
    double mr = O_MAR / 2.0;
    S->nu_max_i = 2.0 * S->ngas * O_ARP_SIG * sqrt(2.0 * O_QE / mr);
    S->lam[SP_E] = S->nu_max_e * P->dt;
    S->lam[SP_I] = S->nu_max_i * P->dt;
    S->p_max_e = 1.0 - exp(-S->lam[SP_E]);
    S->p_max_i = 1.0 - exp(-S->lam[SP_I]);
}

orc_state *orc_create(const orc_params *P, int64_t cap_e, int64_t cap_i, int64_t cap_tp)
{
    orc_state *S = (orc_state *)calloc(1, sizeof(orc_state));
    S->P = *P;
    int N = P->ncell;
    sp_alloc(&S->sp[SP_E], cap_e);
    sp_alloc(&S->sp[SP_I], cap_i);
    sp_alloc(&S->sp[SP_TP], cap_tp);
    S->E = (double *)calloc(N + 1, sizeof(double));
    S->phi = (double *)calloc(N + 1, sizeof(double));
    for (int s = 0; s < 2; s++) {
        S->q[s] = (int64_t *)calloc(N + 1, sizeof(int64_t));
        S->sum_q[s] = (double *)calloc(N + 1, sizeof(double));
        S->sum_flux[s] = (double *)calloc(N + 1, sizeof(double));
        S->iedf[s] = (int64_t *)calloc(NB_IEDF, sizeof(int64_t));
        S->ieadf[s] = (int64_t *)calloc(NB_IEADF_E * NB_ANG, sizeof(int64_t));
        S->sp_e[s] = (int64_t *)calloc(NB_SPE, sizeof(int64_t));
        S->sp_ang[s] = (int64_t *)calloc(NB_ANG, sizeof(int64_t));
    }
    S->sum_phi = (double *)calloc(N + 1, sizeof(double));
    S->tp_dens = (double *)calloc(N + 1, sizeof(double));
    S->tp_vx = (double *)calloc(N + 1, sizeof(double));
    S->tpf_time = (double *)calloc(N, sizeof(double));
    S->tpf_disp = (double *)calloc(N, sizeof(double));
    S->eedf = (int64_t *)calloc(NB_EEDF, sizeof(int64_t));
    derive(S);
    return S;
}

void orc_destroy(orc_state *S)
{
    if (!S) return;
    for (int s = 0; s < 3; s++) sp_free(&S->sp[s]);
    free(S->E); free(S->phi); free(S->sum_phi); free(S->tp_dens); free(S->tp_vx); free(S->eedf);
    free(S->tpf_time); free(S->tpf_disp);
    for (int q = 0; q < 3; q++) { free(S->xs_e[q]); free(S->xs_s[q]); }
    for (int s = 0; s < 2; s++) {
        free(S->q[s]); free(S->sum_q[s]); free(S->sum_flux[s]); free(S->iedf[s]);
        free(S->ieadf[s]); free(S->sp_e[s]); free(S->sp_ang[s]);
    }
    free(S);
}

void orc_derived(const orc_state *S, double out[8])
{
    out[0] = S->ngas; out[1] = S->dx; out[2] = S->nu_max_e; out[3] = S->nu_max_i;
    out[4] = S->p_max_e; out[5] = S->p_max_i; out[6] = S->eps_max; out[7] = lambda_ar_al();
}

/* Initial loading (Sec. "Kinetic Particle Simulation"): positions uniform
 * over the gap, velocities Maxwellian at temperature T (eV), by Box-Muller.
 * The sampled velocity is taken as v^(-1/2).  Ids are tag | k. */
void orc_init_species_range(orc_state *S, int s, int64_t k0, int64_t n, double T_eV);
void orc_init_species(orc_state *S, int s, int64_t n, double T_eV) { orc_init_species_range(S, s, 0, n, T_eV); }

/* the particles k0 .. k0 + n - 1 of the initial loading (ids tag | k): the
 * share of one rank when the particles are split over several */
void orc_init_species_range(orc_state *S, int s, int64_t k0, int64_t n, double T_eV)
{
    orc_sp *p = &S->sp[s];
    double vth = sqrt(T_eV * O_QE / mass_of(s));
    double N = (double)S->P.ncell;
    p->n = 0;
    for (int64_t k = k0; k < k0 + n && k - k0 < p->cap; k++) {
        uint64_t id = TAG[s] | (uint64_t)k;
        uint32_t a[4], b[4];
        draw(S->P.seed, id, 0, PUR_INIT, a);
        draw(S->P.seed, id, 1, PUR_INIT, b);
        double xi = N * (double)(a[0] | 1u) * 0x1p-32;
        double n1, n2, n3, n4;
        box_muller(a[1], a[2], &n1, &n2);
        box_muller(b[0], b[1], &n3, &n4);
        append(S, s, xi, vth * n1, vth * n2, vth * n3, id, 0);
    }
}

/* Replace the analytic cross section of e-Ar process q (0 elastic, 1
 * excitation, 2 ionisation) by a table of n points (n = 0: back to the
 * analytic form); nu_max follows from the tables' largest values, and every
 * electron's next candidate is drawn afresh from the current step (the
 * candidate process is memoryless).  Returns -1 for a bad table. */
int orc_set_cross_section(orc_state *S, int q, int64_t n, const double *E, const double *sg)
{
    if (q < 0 || q > 2 || n < 0 || n == 1) return -1;
    for (int64_t i = 0; i < n; i++)
        if (!(sg[i] >= 0.0) || (i > 0 && !(E[i] > E[i - 1]))) return -1;
    free(S->xs_e[q]); free(S->xs_s[q]);
    S->xs_e[q] = S->xs_s[q] = NULL;
    S->xs_n[q] = n;
    if (n) {
        S->xs_e[q] = (double *)malloc(sizeof(double) * n);
        S->xs_s[q] = (double *)malloc(sizeof(double) * n);
        memcpy(S->xs_e[q], E, sizeof(double) * n);
        memcpy(S->xs_s[q], sg, sizeof(double) * n);
    }
    derive(S);
    orc_sp *p = &S->sp[SP_E];
    for (int64_t k = 0; k < p->n; k++)
        if (p->alive[k]) p->nev[k] = entry_nev(S, SP_E, p->id[k], S->step);
    return 0;
}

/* Load an arbitrary particle set (seeded synthetic inputs in tests). */
int orc_set_species(orc_state *S, int s, int64_t n, const double *xi, const double *vx,
                    const double *vy, const double *vz, const uint64_t *id)
{
    orc_sp *p = &S->sp[s];
    if (n > p->cap) return -1;
    p->n = 0;
    for (int64_t k = 0; k < n; k++) append(S, s, xi[k], vx[k], vy[k], vz[k], id[k], S->step);
    for (int64_t k = 0; k < n; k++) p->alive[k] = xi[k] >= 0.0;
    return 0;
}

/* Copy out the alive particles (index order). Returns the number copied. */
int64_t orc_get_species(const orc_state *S, int s, int64_t cap, double *xi, double *vx,
                        double *vy, double *vz, uint64_t *id)
{
    const orc_sp *p = &S->sp[s];
    int64_t m = 0;
    for (int64_t k = 0; k < p->n; k++) {
        if (!p->alive[k]) continue;
        if (m < cap) {
            xi[m] = p->xi[k]; vx[m] = p->vx[k]; vy[m] = p->vy[k]; vz[m] = p->vz[k]; id[m] = p->id[k];
        }
        m++;
    }
    return m;
}

/* deposit + solve for the current state at the current step (creation) */
void orc_field(orc_state *S) { field_for_step(S, S->step); }

void orc_get_field(const orc_state *S, double *E, double *phi, int64_t *q_e, int64_t *q_i)
{
    int N = S->P.ncell;
    memcpy(E, S->E, sizeof(double) * (N + 1));
    memcpy(phi, S->phi, sizeof(double) * (N + 1));
    memcpy(q_e, S->q[SP_E], sizeof(int64_t) * (N + 1));
    memcpy(q_i, S->q[SP_I], sizeof(int64_t) * (N + 1));
}

void orc_set_field(orc_state *S, const double *E)
{
    memcpy(S->E, E, sizeof(double) * (S->P.ncell + 1));
}

void orc_counters(const orc_state *S, int64_t *out)
{
    for (int c = 0; c < C_NCOUNT; c++) out[c] = S->cnt[c];
    for (int s = 0; s < 3; s++) {
        int64_t a = 0;
        for (int64_t k = 0; k < S->sp[s].n; k++) a += S->sp[s].alive[k];
        out[C_NE + s] = a;
    }
}

/* ======================= the PIC/MCC step ================================ */
/* bin of x on [0, xmax) in nb bins; below the range the first bin, at or
 * above it the last (the scaled value is clamped before the conversion) */
/* Integers decided by floating point (a histogram bin, the process of a
 * collision, a sputter trial, the partner and the acceptance of a TP
 * candidate) are decided in FP32, the precision of the GPU path's kinematics,
 * on the oracle's FP64 operands rounded to FP32; everything else stays FP64. */
static int bin_of(double x, double xmax, int nb)
{
    float t = (float)x / (float)xmax * (float)nb;
    if (!(t < (float)nb)) return nb - 1;
    if (!(t >= 0.0f)) return 0;
    return (int)t;
}

/* 1-degree bin of a polar angle given in degrees */
static int ang_bin(double deg)
{
    float t = (float)deg;
    if (!(t < (float)NB_ANG)) return NB_ANG - 1;
    if (!(t >= 0.0f)) return 0;
    return (int)t;
}

static void hist_add(int64_t *h, int nb, double x, double xmax)
{
    h[bin_of(x, xmax, nb)]++;
}

/* sputter launch at an ion impact (Sec. "Wall Interactions" of the TPM):
 * Y(E) = 0.1 sqrt(E/30 eV - 1) above 30 eV, N = ceil(Y) trials, each
 * succeeding when R <= Y/N; each success inserts an atom at the impact
 * point with a Thompson energy and a cosine angle, aimed into the gap. */
static void sputter(orc_state *S, uint64_t ion_id, uint32_t l, double E, int electrode)
{
    double Y = orc_yield(E);
    if (Y <= 0.0) return;
    int Nt = (int)ceil(Y);
    if (Nt > O_SP_MAXN) Nt = O_SP_MAXN;
    double Emax = lambda_ar_al() * E;
    double N = (double)S->P.ncell;
    for (int k = 0; k < Nt; k++) {
        uint32_t t[4];
        draw(S->P.seed, ion_id, l, PUR_SP_TRIAL + (k >> 2), t);
        if (!((float)u23(t[k & 3]) <= (float)Y / (float)Nt)) continue;
        uint32_t ce[4], ci[4];
        draw(S->P.seed, ion_id, l, PUR_SP_EMIT + k, ce);
        draw(S->P.seed, ion_id, l, PUR_SP_ID + k, ci);
        double v[3];
        orc_emit(u23(ce[0]), u23(ce[1]), u23(ce[2]), Emax, electrode == 0 ? 1.0 : -1.0, v);
        double xi = electrode == 0 ? N * 0x1p-32 : N * (1.0 - 0x1p-32);
        if (append(S, SP_TP, xi, v[0], v[1], v[2], child_id(ci[0], ci[1], SP_TP), 0) >= 0)
            S->cnt[electrode == 0 ? C_SPUT_L : C_SPUT_R]++;
    }
}

/* electron null-collision MCC for one particle (Sec. "Particle Collisions") */
static void mcc_electron(orc_state *S, int64_t k, uint32_t l)
{
    orc_sp *p = &S->sp[SP_E];
    uint32_t c[4];
    if (S->P.coll_mode == 1) {                               /* the literal per-step test */
        draw(S->P.seed, p->id[k], l, PUR_COLL, c);
        if (!(u23(c[0]) < S->p_max_e)) return;               /* not a candidate */
    } else {
        if (p->nev[k] != l) return;                          /* not a candidate */
        uint32_t cg[4];
        draw(S->P.seed, p->id[k], l, PUR_COLL, c);
        draw(S->P.seed, p->id[k], l, PUR_GAP, cg);
        p->nev[k] = l + orc_gap(S->lam[SP_E], cg[0]);
    }
    double v2 = p->vx[k] * p->vx[k] + p->vy[k] * p->vy[k] + p->vz[k] * p->vz[k];
    double v = sqrt(v2);
    double eps = 0.5 * O_ME * v2 / O_QE;
    if (eps > S->eps_max) S->cnt[C_NUMERICS]++;
    double sg[3];
    electron_sigma(S, eps, sg);
    double nu_el = S->ngas * sg[0] * v;
    double nu_exc = S->ngas * sg[1] * v;
    double nu_ion = S->ngas * sg[2] * v;
    float r = (float)u23(c[1]) * (float)S->nu_max_e;        /* the process, in FP32 */
    float f_el = (float)nu_el, f_exc = (float)nu_exc, f_ion = (float)nu_ion;
    double d[3];
    iso_dir(c[2], c[3], d);
    if (r < f_el) {
        double cchi = v > 0.0 ? (d[0] * p->vx[k] + d[1] * p->vy[k] + d[2] * p->vz[k]) / v : 1.0;
        double fac = 1.0 - (2.0 * O_ME / O_MAR) * (1.0 - cchi);
        double vn = v * sqrt(fac);
        p->vx[k] = vn * d[0]; p->vy[k] = vn * d[1]; p->vz[k] = vn * d[2];
        S->cnt[C_ELASTIC]++;
    } else if (r < f_el + f_exc) {
        double vn = sqrt(2.0 * (eps - O_EXC_TH) * O_QE / O_ME);
        p->vx[k] = vn * d[0]; p->vy[k] = vn * d[1]; p->vz[k] = vn * d[2];
        S->cnt[C_EXCIT]++;
    } else if (r < f_el + f_exc + f_ion) {
        double epr = eps - O_ION_TH;
        uint32_t ci[4], cn[4], cb[4];
        draw(S->P.seed, p->id[k], l, PUR_IONIZE, ci);
        draw(S->P.seed, p->id[k], l, PUR_NEWION, cn);
        draw(S->P.seed, p->id[k], l, PUR_BIRTH_ID, cb);
        double e_ej = u23(ci[0]) * epr;
        double e_sc = epr - e_ej;
        double vs = sqrt(2.0 * e_sc * O_QE / O_ME);
        double ve = sqrt(2.0 * e_ej * O_QE / O_ME);
        double d2[3];
        iso_dir(ci[1], ci[2], d2);
        double n1, n2, n3, n4;
        box_muller(cn[0], cn[1], &n1, &n2);
        box_muller(cn[2], cn[3], &n3, &n4);
        double vg = sqrt(O_KB * S->P.Tg / O_MAR);
        double xi = p->xi[k];
        p->vx[k] = vs * d[0]; p->vy[k] = vs * d[1]; p->vz[k] = vs * d[2];
        append(S, SP_E, xi, ve * d2[0], ve * d2[1], ve * d2[2], child_id(cb[0], cb[1], SP_E), l + 1);
        append(S, SP_I, xi, vg * n1, vg * n2, vg * n3, child_id(cb[2], cb[3], SP_I), l + 1);
        S->cnt[C_IONIZ]++;
    }
}

/* Ar+ null-collision MCC with a thermal gas partner (Sec. "Kinetic Particle
 * Simulation": v_r = |v - v_bg|, v_bg Maxwellian; Sec. "Particle Collisions") */
static void mcc_ion(orc_state *S, int64_t k, uint32_t l)
{
    orc_sp *p = &S->sp[SP_I];
    uint32_t c[4];
    if (S->P.coll_mode == 1) {                               /* the literal per-step test */
        draw(S->P.seed, p->id[k], l, PUR_COLL, c);
        if (!(u23(c[0]) < S->p_max_i)) return;               /* not a candidate */
    } else {
        if (p->nev[k] != l) return;                          /* not a candidate */
        uint32_t cn[4];
        draw(S->P.seed, p->id[k], l, PUR_COLL, c);
        draw(S->P.seed, p->id[k], l, PUR_GAP, cn);
        p->nev[k] = l + orc_gap(S->lam[SP_I], cn[0]);
    }
    uint32_t cg[4];
    draw(S->P.seed, p->id[k], l, PUR_GAS, cg);
    double n1, n2, n3, n4;
    box_muller(cg[0], cg[1], &n1, &n2);
    box_muller(cg[2], cg[3], &n3, &n4);
    double vg = sqrt(O_KB * S->P.Tg / O_MAR);
    double w[3] = {vg * n1, vg * n2, vg * n3};
    double g[3] = {p->vx[k] - w[0], p->vy[k] - w[1], p->vz[k] - w[2]};
    double gm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    double mr = O_MAR / 2.0;
    double eps = 0.5 * mr * gm * gm / O_QE;
    double nu_cx = gm > 0.0 ? S->ngas * orc_sigma_i(eps) * gm : 0.0;
    double nu_iso = nu_cx;
    double r = u23(c[1]) * S->nu_max_i;
    if (r < nu_cx) {
        p->vx[k] = w[0]; p->vy[k] = w[1]; p->vz[k] = w[2];
        S->cnt[C_CX]++;
    } else if (r < nu_cx + nu_iso) {
        double d[3];
        iso_dir(c[2], c[3], d);
        double v0[3] = {p->vx[k], p->vy[k], p->vz[k]};
        p->vx[k] = 0.5 * (v0[0] + w[0]) + 0.5 * gm * d[0];
        p->vy[k] = 0.5 * (v0[1] + w[1]) + 0.5 * gm * d[1];
        p->vz[k] = 0.5 * (v0[2] + w[2]) + 0.5 * gm * d[2];
        S->cnt[C_ISO]++;
    }
}

static void wall_ion(orc_state *S, int64_t k, uint32_t l, int electrode)
{
    orc_sp *p = &S->sp[SP_I];
    double v2 = p->vx[k] * p->vx[k] + p->vy[k] * p->vy[k] + p->vz[k] * p->vz[k];
    double E = 0.5 * O_MAR * v2 / O_QE;
    double ct = v2 > 0.0 ? fabs(p->vx[k]) / sqrt(v2) : 1.0;
    if (ct > 1.0) ct = 1.0;
    double th = acos(ct) * 180.0 / O_PI;
    double emax = S->P.V0 > 0.0 ? 2.0 * S->P.V0 : 1.0;   /* [0, 2 V0]; [0, 1 eV] without a source */
    hist_add(S->iedf[electrode], NB_IEDF, E, emax);
    int be = bin_of(E, emax, NB_IEADF_E);
    S->ieadf[electrode][be * NB_ANG + ang_bin(th)]++;
    S->cnt[electrode == 0 ? C_IMP_I_L : C_IMP_I_R]++;
    if (S->P.sputter) sputter(S, p->id[k], l, E, electrode);
}

void orc_tp_step(orc_state *S, int64_t nsteps, double dt_tp);
static double gamma_mt(double k, uint64_t seed, uint64_t id, uint32_t e, uint32_t base);

/* One PIC/MCC cycle l -> l+1 for both charged species (Fig. 4 order: the
 * field E^l is already known; interpolate, push (leapfrog, Eqs. for r and
 * v), walls, collisions; then charge assignment and field solve for l+1). */
/* One PIC/MCC cycle in two halves.  orc_step_particles: interpolation, push,
 * walls and collisions of every particle and the charge assignment of
 * x^{l+1} into q; orc_step_field: the field solve of step l+1 from q, the
 * time averages and the coupled TP step.  Between the two a caller that
 * holds only a share of the particles (the particles split over several
 * ranks) replaces q by the sum over the ranks (orc_set_deposit). */
void orc_step_particles(orc_state *S)
{
    uint32_t l = S->step;
    int N = S->P.ncell;
    double dx = S->dx;
    int64_t n_start[2] = {S->sp[SP_E].n, S->sp[SP_I].n};   /* births of this step wait */
    for (int s = 0; s < 2; s++) {
        orc_sp *p = &S->sp[s];
        double qm = charge_of(s) / mass_of(s);
        int64_t n0 = n_start[s];
        for (int64_t k = 0; k < n0; k++) {
            if (!p->alive[k]) continue;
            /* field interpolation (Sec. "Field Interpolation") */
            double j = floor(p->xi[k]);
            double f = p->xi[k] - j;
            int m = (int)j;
            double Ek = (1.0 - f) * S->E[m] + f * S->E[m + 1];
            /* leapfrog (Eqs. pushinv, pushinr) */
            p->vx[k] = p->vx[k] + qm * Ek * S->P.dt;
            p->xi[k] = p->xi[k] + p->vx[k] * S->P.dt / dx;
            /* wall interaction (Sec. "Wall Interaction"): absorb */
            if (p->xi[k] <= 0.0 || p->xi[k] >= (double)N) {
                int el = p->xi[k] <= 0.0 ? 0 : 1;
                p->alive[k] = 0;
                if (s == SP_E) S->cnt[el == 0 ? C_IMP_E_L : C_IMP_E_R]++;
                else wall_ion(S, k, l, el);
                continue;
            }
            /* collisions */
            if (s == SP_E) mcc_electron(S, k, l);
            else mcc_ion(S, k, l);
        }
    }
    S->step = l + 1;
    deposit_all(S);
}

void orc_step_field(orc_state *S)
{
    int N = S->P.ncell;
    solve_for_step(S, S->step);
    /* time averages (Sec. "Kinetic Particle Simulation": averaging) */
    for (int m = 0; m <= N; m++) {
        S->sum_q[0][m] += (double)S->q[0][m];
        S->sum_q[1][m] += (double)S->q[1][m];
        S->sum_phi[m] += S->phi[m];
    }
    S->n_avg++;
    if (S->P.diag_every > 0 && S->step % (uint32_t)S->P.diag_every == 0) {
        for (int s = 0; s < 2; s++) {
            orc_sp *p = &S->sp[s];
            for (int64_t k = 0; k < p->n; k++) {
                if (!p->alive[k]) continue;
                double j = floor(p->xi[k]);
                double f = p->xi[k] - j;
                int m = (int)j;
                S->sum_flux[s][m] += (1.0 - f) * p->vx[k];
                S->sum_flux[s][m + 1] += f * p->vx[k];
                if (s == SP_E && p->xi[k] >= 0.45 * N && p->xi[k] < 0.55 * N) {
                    double v2 = p->vx[k] * p->vx[k] + p->vy[k] * p->vy[k] + p->vz[k] * p->vz[k];
                    hist_add(S->eedf, NB_EEDF, 0.5 * O_ME * v2 / O_QE, 64.0);
                }
            }
        }
        S->n_flux++;
    }
    if (S->P.sputter && S->P.tp_every > 0 && S->step % (uint32_t)S->P.tp_every == 0)
        orc_tp_step(S, 1, S->P.tp_every * S->P.dt);
}

static void pic_one_step(orc_state *S)
{
    orc_step_particles(S);
    orc_step_field(S);
}

/* the field solve of the current step from the deposit held (after
 * orc_set_deposit at creation) */
void orc_solve(orc_state *S) { solve_for_step(S, S->step); }

/* the charge assignment the next field solve uses (int64[N+1] each) */
void orc_set_deposit(orc_state *S, const int64_t *q_e, const int64_t *q_i)
{
    memcpy(S->q[SP_E], q_e, sizeof(int64_t) * (S->P.ncell + 1));
    memcpy(S->q[SP_I], q_i, sizeof(int64_t) * (S->P.ncell + 1));
}

void orc_step(orc_state *S, int64_t nsteps)
{
    for (int64_t i = 0; i < nsteps; i++) pic_one_step(S);
}

/* ======================= test particles ================================== */
/* ======================= TP collision models ============================= */
/* Sec. "Binary Interactions": hard spheres (sigma_tp), the variable hard
 * sphere model, sigma_T(g) = pi b_max(g)^2 with b_max from Eq.
 * maximumimpactparameter for the Al-Ar pair (reduced mass m_r, reference
 * diameter and viscosity index of the pair), and the M1 model, which uses
 * the VHS law with d_ref,M1 = sqrt(4/3) d_ref,VHS.  Both VHS forms give
 * sigma(g) g = K g^alpha with alpha = 2 - 2 omega. */
static double tp_mr(void) { return O_MAL * O_MAR / (O_MAL + O_MAR); }

double orc_tp_sigma(const orc_state *S, double g)
{
    const orc_params *P = &S->P;
    if (P->tp_model == 0) return P->sigma_tp;
    double d = P->tp_model == 2 ? sqrt(4.0 / 3.0) * P->dref : P->dref;
    double b2 = d * d * pow(2.0 * O_KB * P->tref / (tp_mr() * g * g), P->omega - 0.5) / tgamma(2.5 - P->omega);
    return O_PI * b2;
}

/* reference diameter from the viscosity mu_ref at T_ref (Eq. referencediameter) */
double orc_vhs_dref(double mu_ref, double t_ref, double omega, double mass)
{
    return sqrt(15.0 * sqrt(mass * O_KB * t_ref / O_PI) / (8.0 * (2.5 - omega) * (3.5 - omega) * mu_ref));
}

/* Direction of the post-collision relative velocity for a scattering draw
 * (r1, r2): hard spheres and VHS scatter isotropically in the centre-of-mass
 * frame; M1 turns g by chi = pi (1 - b / b_max) with b = b_max sqrt(r1),
 * at the azimuth eps = 2 pi r2 about g (the frame of g: e1 along g x x^, or
 * g x y^ when |g_x| >= 0.9 |g|, e2 = g^ x e1). */
void orc_tp_scatter(int model, const double g[3], uint32_t r1, uint32_t r2, double out[3])
{
    double gm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (model != 2 || gm == 0.0) {
        iso_dir(r1, r2, out);
        return;
    }
    double u[3] = {g[0] / gm, g[1] / gm, g[2] / gm};
    double a[3] = {0.0, 0.0, 0.0};
    if (fabs(u[0]) < 0.9) a[0] = 1.0; else a[1] = 1.0;
    double e1[3] = {u[1] * a[2] - u[2] * a[1], u[2] * a[0] - u[0] * a[2], u[0] * a[1] - u[1] * a[0]};
    double n1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int i = 0; i < 3; i++) e1[i] /= n1;
    double e2[3] = {u[1] * e1[2] - u[2] * e1[1], u[2] * e1[0] - u[0] * e1[2], u[0] * e1[1] - u[1] * e1[0]};
    double chi = O_PI * (1.0 - sqrt(u23(r1)));
    double eps = 2.0 * O_PI * u23(r2);
    double cc = cos(chi), sc = sin(chi), ce = cos(eps), se = sin(eps);
    for (int i = 0; i < 3; i++) out[i] = cc * u[i] + sc * (ce * e1[i] + se * e2[i]);
}

/* One TP step (Sec. "Test Particle Method"): free flight x += v_x dt, sticking
 * at either wall with the absorbed flux recorded, and a binary collision with
 * a partner w from the Maxwellian gas with probability p(g) = 1 - exp(-n
 * sigma(g) g dt), g = |v - w| (Eq. collisionprobability1 with tau_c = 1/(n
 * sigma(g) g)); scattering in the centre-of-mass frame (orc_tp_scatter).
 *
 * tp_mode 1 is the method as the paper states it: every step draws a partner
 * (PUR_TP_GAS) and the test word (PUR_TP_COLL word 0).
 *
 * tp_mode 0 takes the same per-step law in two parts, as the null-collision
 * method does for the charged particles (Sec. "Particle Collisions"):
 *  - With sigma(g) g = K g^alpha (hard spheres: K = sigma, alpha = 1; VHS and
 *    M1: alpha = 2 - 2 omega <= 1), p(g) <= n K dt g^alpha <= n K dt
 *    (|v|^alpha + |w|^alpha).  So every step is a candidate with the
 *    probability P^ = n K dt (|v|^alpha + <|w|^alpha>), independently of the
 *    other steps, and the steps between candidates are geometric.
 *    P^ is that bound rounded up to 8 significant bits (tp_cand_prob).
 *  - A candidate draws one partner from (|v|^alpha + |w|^alpha) f(w) / (|v|^alpha
 *    + <|w|^alpha>) -- a Maxwellian w with probability |v|^alpha / (|v|^alpha +
 *    <|w|^alpha>), else |w|^2/c^2 ~ Gamma((3 + alpha)/2) in an isotropic
 *    direction -- and collides with probability p(g) (|v|^alpha +
 *    <|w|^alpha>) / (P^ (|v|^alpha + |w|^alpha)) <= 1 (PUR_TP_CAND,
 *    PUR_TP_CAND + 1 word 1).
 *  - P^ times the proposal density times that probability is f(w) p(g): the
 *    law of the literal test.  |v| changes only at a collision, so the next
 *    gap is drawn at the current |v| after each candidate (PUR_TP_GAP); an
 *    atom's first gap is drawn at the first step that moves it (PUR_TP_GAP0).
 *  - nev holds the next candidate step plus one (0: none drawn yet; a step
 *    index below the current one, left by the event-driven flight, is
 *    redrawn the same way).  The scattering uses PUR_TP_COLL words 1, 2 as
 *    in tp_mode 1.  It needs P^ <= 1 (dt << tau_c, Sec. "Limitations and
 *    Constraints"); a larger P^ counts as NUMERICS. */

/* TP steps from one candidate to the next at the per-step probability Ph:
 * geometric, by inversion, 1 + floor(ln R / ln(1 - Ph)) */
uint32_t orc_tp_gap(double Ph, uint32_t w)
{
    if (!(Ph < 1.0)) return 1u;
    if (!(Ph > 0.0)) return 2147483647u;
    double x = log(u23(w)) / log1p(-Ph);
    if (!(x < 2147483646.0)) return 2147483647u;
    return 1u + (uint32_t)floor(x);
}

/* <|w|^alpha> of the Maxwellian gas of most probable speed c */
static double gas_mean_pow(double c, double alpha)
{
    return pow(c, alpha) * tgamma(0.5 * (3.0 + alpha)) / tgamma(1.5);
}

/* x rounded up to 8 significant bits (0, NaN and infinity unchanged) */
static double round_up8(double x)
{
    if (!(x > 0.0) || isinf(x)) return x;
    int e;
    double m = frexp(x, &e);
    return ldexp(ceil(m * 256.0) / 256.0, e);
}

/* The candidate probability per step P^ of an atom of speed vm: the bound
 * n K dt (|v|^alpha + <|w|^alpha>) rounded up to 8 significant bits.  Any
 * larger value is a majorant too (the acceptance below carries the ratio),
 * and the rounding lets implementations that evaluate the bound in other
 * precisions reach the same P^, hence the same gaps. */
static double tp_cand_prob(const orc_state *S, double vm, double dt_tp)
{
    double c = sqrt(2.0 * O_KB * S->P.Tg / O_MAR);
    double alpha = S->P.tp_model == 0 ? 1.0 : 2.0 - 2.0 * S->P.omega;
    double K = S->P.tp_model == 0 ? S->P.sigma_tp : orc_tp_sigma(S, 1.0);
    return round_up8(S->ngas * K * dt_tp * (pow(vm, alpha) + gas_mean_pow(c, alpha)));
}

/* one candidate of tp_mode 0 at step s: returns 1 and the partner w when it
 * is a real collision */
static int tp_candidate(orc_state *S, uint64_t id, uint32_t s, const double v[3], double dt_tp, double w[3])
{
    double c = sqrt(2.0 * O_KB * S->P.Tg / O_MAR);
    double alpha = S->P.tp_model == 0 ? 1.0 : 2.0 - 2.0 * S->P.omega;
    double K = S->P.tp_model == 0 ? S->P.sigma_tp : orc_tp_sigma(S, 1.0);
    double b = S->ngas * K * dt_tp;
    double vm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double va = pow(vm, alpha), ma = gas_mean_pow(c, alpha);
    uint32_t a[4], e[4];
    draw(S->P.seed, id, s, PUR_TP_CAND, a);
    draw(S->P.seed, id, s, PUR_TP_CAND + 1, e);
    if ((float)u23(a[0]) * ((float)va + (float)ma) < (float)va) {   /* the partner's law, in FP32 */
        double vg = c / sqrt(2.0), n1, n2, n3, n4;
        box_muller(a[1], a[2], &n1, &n2);
        box_muller(a[3], e[0], &n3, &n4);
        w[0] = vg * n1; w[1] = vg * n2; w[2] = vg * n3;
    } else {
        double x2 = S->P.tp_model == 0 ? -log(u23(a[1]) * u23(a[2]))
                                       : gamma_mt(0.5 * (3.0 + alpha), S->P.seed, id, s, PUR_TP_GAMMA);
        double sp = c * sqrt(x2), d[3];
        iso_dir(a[3], e[0], d);
        w[0] = sp * d[0]; w[1] = sp * d[1]; w[2] = sp * d[2];
    }
    double g = sqrt((v[0] - w[0]) * (v[0] - w[0]) + (v[1] - w[1]) * (v[1] - w[1]) + (v[2] - w[2]) * (v[2] - w[2]));
    double wm = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    /* accept with p(g) (|v|^alpha + <|w|^alpha>) / (P^ (|v|^alpha + |w|^alpha)) */
    double Ph = tp_cand_prob(S, vm, dt_tp);
    float acc_l = (float)u23(e[1]) * (float)Ph * ((float)va + (float)pow(wm, alpha));   /* in FP32 */
    float acc_r = ((float)va + (float)ma) * (float)(-expm1(-b * pow(g, alpha)));
    return acc_l < acc_r;
}

void orc_tp_step(orc_state *S, int64_t nsteps, double dt_tp)
{
    orc_sp *p = &S->sp[SP_TP];
    int N = S->P.ncell;
    double dx = S->dx;
    double vg = sqrt(O_KB * S->P.Tg / O_MAR);
    double mu = O_MAL + O_MAR;
    int geo = S->P.tp_mode == 0;
    if (geo && dt_tp != S->tp_gap_dt) {          /* gaps drawn for another dt: redraw them all */
        for (int64_t k = 0; k < p->n; k++) p->nev[k] = 0;
        S->tp_gap_dt = dt_tp;
    }
    for (int64_t it = 0; it < nsteps; it++) {
        uint32_t s = S->tp_step;
        for (int64_t k = 0; k < p->n; k++) {
            if (!p->alive[k]) continue;
            p->xi[k] = p->xi[k] + p->vx[k] * dt_tp / dx;
            if (p->xi[k] <= 0.0 || p->xi[k] >= (double)N) {
                int el = p->xi[k] <= 0.0 ? 0 : 1;
                double v2 = p->vx[k] * p->vx[k] + p->vy[k] * p->vy[k] + p->vz[k] * p->vz[k];
                double E = 0.5 * O_MAL * v2 / O_QE;
                double ct = v2 > 0.0 ? fabs(p->vx[k]) / sqrt(v2) : 1.0;
                if (ct > 1.0) ct = 1.0;
                hist_add(S->sp_e[el], NB_SPE, E, 300.0);
                S->sp_ang[el][ang_bin(acos(ct) * 180.0 / O_PI)]++;
                S->cnt[el == 0 ? C_TPDEP_L : C_TPDEP_R]++;
                p->alive[k] = 0;
                continue;
            }
            double v[3] = {p->vx[k], p->vy[k], p->vz[k]};
            double w[3], g[3];
            int hit;
            if (geo) {
                uint32_t nv = p->nev[k];
                if (nv == 0u || (int32_t)(nv - 1u - s) < 0) {       /* first gap of this atom */
                    uint32_t r[4];
                    draw(S->P.seed, p->id[k], s, PUR_TP_GAP0, r);
                    double Ph = tp_cand_prob(S, sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]), dt_tp);
                    if (!(Ph <= 1.0)) S->cnt[C_NUMERICS]++;
                    nv = s + orc_tp_gap(Ph, r[0]);
                    p->nev[k] = nv;
                }
                if (nv - 1u != s) continue;                           /* not a candidate */
                hit = tp_candidate(S, p->id[k], s, v, dt_tp, w);
            } else {
                uint32_t cg[4], cc0[4];
                draw(S->P.seed, p->id[k], s, PUR_TP_GAS, cg);
                double n1, n2, n3, n4;
                box_muller(cg[0], cg[1], &n1, &n2);
                box_muller(cg[2], cg[3], &n3, &n4);
                w[0] = vg * n1; w[1] = vg * n2; w[2] = vg * n3;
                double gx = v[0] - w[0], gy = v[1] - w[1], gz = v[2] - w[2];
                double gm0 = sqrt(gx * gx + gy * gy + gz * gz);
                double sig = gm0 > 0.0 ? orc_tp_sigma(S, gm0) : 0.0;
                double P = 1.0 - exp(-S->ngas * sig * gm0 * dt_tp);
                draw(S->P.seed, p->id[k], s, PUR_TP_COLL, cc0);
                hit = (float)u23(cc0[0]) < (float)P;               /* in FP32 */
            }
            if (hit) {
                uint32_t cc[4];
                draw(S->P.seed, p->id[k], s, PUR_TP_COLL, cc);
                for (int i = 0; i < 3; i++) g[i] = v[i] - w[i];
                double gm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
                double d[3];
                orc_tp_scatter(S->P.tp_model, g, cc[1], cc[2], d);
                double vc[3] = {(O_MAL * v[0] + O_MAR * w[0]) / mu, (O_MAL * v[1] + O_MAR * w[1]) / mu,
                                (O_MAL * v[2] + O_MAR * w[2]) / mu};
                p->vx[k] = vc[0] + (O_MAR / mu) * gm * d[0];
                p->vy[k] = vc[1] + (O_MAR / mu) * gm * d[1];
                p->vz[k] = vc[2] + (O_MAR / mu) * gm * d[2];
                S->cnt[C_TPCOLL]++;
            }
            if (geo) {                                                /* the next candidate */
                uint32_t r[4];
                draw(S->P.seed, p->id[k], s, PUR_TP_GAP, r);
                double vm = sqrt(p->vx[k] * p->vx[k] + p->vy[k] * p->vy[k] + p->vz[k] * p->vz[k]);
                double Ph = tp_cand_prob(S, vm, dt_tp);
                if (!(Ph <= 1.0)) S->cnt[C_NUMERICS]++;
                p->nev[k] = s + 1u + orc_tp_gap(Ph, r[0]);
            }
        }
        /* grid moments of the TP density and mean velocity (Sec. "Limitations
         * and Constraints" of the TPM: cell-based averages), sampled every
         * diag_every TP steps */
        int samp = S->P.diag_every > 0 && (s + 1) % (uint32_t)S->P.diag_every == 0;
        for (int64_t k = 0; samp && k < p->n; k++) {
            if (!p->alive[k]) continue;
            double j = floor(p->xi[k]);
            double f = p->xi[k] - j;
            int m = (int)j;
            S->tp_dens[m] += 1.0 - f;
            S->tp_dens[m + 1] += f;
            S->tp_vx[m] += (1.0 - f) * p->vx[k];
            S->tp_vx[m + 1] += f * p->vx[k];
        }
        if (samp) S->n_tp_samp++;
        S->tp_step = s + 1;
    }
}

/* ======================= event-driven TP flight ========================== */
/* The gridless alternative of Sec. "Kinetic Particle Simulation" (free
 * flight) and Sec. "Limitations and Constraints" (time-weighted densities):
 * instead of testing for a collision every dt, each atom flies straight for
 * a free-flight time tau = -tau_c ln R_f, tau_c = 1/nu, to its next
 * collision or to a wall.  For hard spheres (sigma constant) in a Maxwellian
 * gas the rate is nu(v) = n sigma <|v - w|>, the relative speed averaged over
 * the gas (closed form below), and at a collision the partner w has the
 * density |v - w| f(w) / <|v - w|>: the collision law of the per-step test
 * of orc_tp_step in the limit dt -> 0.  With the VHS and M1 models
 * (sigma(g) g = K g^alpha) the flight runs at a majorant rate and each
 * candidate is a real collision or a null event (thinning); null events count
 * as events.  Random words of event e of an atom:
 * Philox(id, e, TPF_FLIGHT), (id, e, TPF_PARTNER + 2t [+1]) for proposal t,
 * (id, e, TPF_SCATTER); e is kept per atom (orc_sp.nev).  Residence time and
 * signed path length are added per cell for each straight segment. */

/* <|v - w|> for a particle of speed v in a Maxwellian gas of most probable
 * speed c: c [(s + 1/(2s)) erf(s) + exp(-s^2)/sqrt(pi)], s = v/c (kinetic
 * theory of the mean relative speed); its series 2c/sqrt(pi) (1 + s^2/3) for
 * s < 1e-3. */
double orc_mean_rel_speed(double v, double c)
{
    double s = v / c;
    if (s < 1e-3) return 2.0 * c / sqrt(O_PI) * (1.0 + s * s / 3.0);
    return c * ((s + 0.5 / s) * erf(s) + exp(-s * s) / sqrt(O_PI));
}

/* Partner of a collision of an atom with velocity v: rejection from the
 * proposal (|v| + |w|) f(w), drawn as a mixture -- with probability |v| /
 * (|v| + <|w|>) a Maxwellian w, otherwise a Maxwellian weighted by |w|
 * (|w|^2/c^2 ~ Gamma(2), i.e. -ln(R1 R2), direction isotropic) -- and accepted
 * with probability |v - w| / (|v| + |w|) <= 1.  Returns the proposals used
 * (TPF_TRIES + 1 if none was accepted: w is then the last proposal). */
int orc_tpf_partner(uint64_t seed, uint64_t id, uint32_t e, double Tg, const double v[3], double w[3])
{
    double c = sqrt(2.0 * O_KB * Tg / O_MAR);
    double vg = c / sqrt(2.0);
    double vm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double mw = 2.0 * c / sqrt(O_PI);
    for (int t = 0; t < TPF_TRIES; t++) {
        uint32_t a[4], b[4];
        draw(seed, id, e, PUR_TPF_PARTNER + 2 * t, a);
        draw(seed, id, e, PUR_TPF_PARTNER + 2 * t + 1, b);
        if ((float)u23(a[0]) * ((float)vm + (float)mw) < (float)vm) {   /* in FP32 */
            double n1, n2, n3, n4;
            box_muller(a[1], a[2], &n1, &n2);
            box_muller(a[3], b[0], &n3, &n4);
            w[0] = vg * n1; w[1] = vg * n2; w[2] = vg * n3;
        } else {
            double sp = c * sqrt(-log(u23(a[1]) * u23(a[2])));
            double d[3];
            iso_dir(a[3], b[0], d);
            w[0] = sp * d[0]; w[1] = sp * d[1]; w[2] = sp * d[2];
        }
        double g[3] = {v[0] - w[0], v[1] - w[1], v[2] - w[2]};
        double gm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        double wm = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        if ((float)u23(b[1]) * ((float)vm + (float)wm) < (float)gm) return t + 1;   /* in FP32 */
    }
    return TPF_TRIES + 1;
}

/* Gamma variate of shape k >= 1 (Marsaglia and Tsang, ACM TOMS 26, 2000):
 * d = k - 1/3, x normal, v = (1 + x/sqrt(9d))^3, accepted when
 * ln U < x^2/2 + d - d v + d ln v; attempt t draws (id, e, TPF_GAMMA + t). */
static double gamma_mt(double k, uint64_t seed, uint64_t id, uint32_t e, uint32_t base)
{
    double d = k - 1.0 / 3.0, cc = 1.0 / sqrt(9.0 * d);
    for (int t = 0; t < TPF_GAMMA_TRIES; t++) {
        uint32_t r[4];
        draw(seed, id, e, base + t, r);
        double x, unused;
        box_muller(r[0], r[1], &x, &unused);
        double v = 1.0 + cc * x;
        if (v <= 0.0) continue;
        v = v * v * v;
        if ((float)log(u23(r[2])) < (float)(0.5 * x * x + d - d * v + d * log(v))) return d * v;   /* in FP32 */
    }
    return d;
}

/* residence time and signed path of the straight segment xi0 -> xi1 (cell
 * units) flown at v_x over tau seconds, cell by cell */
static void tpf_segment(orc_state *S, double xi0, double xi1, double vx, double tau)
{
    int N = S->P.ncell;
    double dx = S->dx;
    if (vx == 0.0 || xi0 == xi1) {
        int j = (int)floor(xi0);
        if (j > N - 1) j = N - 1;
        if (j < 0) j = 0;
        S->tpf_time[j] += tau;
        return;
    }
    double lo = fmin(xi0, xi1), hi = fmax(xi0, xi1);
    int j0 = (int)floor(lo), j1 = (int)floor(hi);
    if (j1 > N - 1) j1 = N - 1;
    for (int j = j0; j <= j1; j++) {
        double ov = fmin(hi, (double)(j + 1)) - fmax(lo, (double)j);
        if (ov <= 0.0) continue;
        S->tpf_time[j] += ov * dx / fabs(vx);
        S->tpf_disp[j] += (vx > 0.0 ? ov : -ov) * dx;
    }
}

/* Run every live TP atom through at most max_events flight events (in
 * index order, atom by atom): flight to the next collision or to a wall,
 * sticking there with the absorbed flux recorded, else a hard-sphere
 * collision with a partner from the gas, isotropic in the centre-of-mass
 * frame.  Returns the atoms still alive. */
int64_t orc_tp_flight(orc_state *S, int64_t max_events)
{
    orc_sp *p = &S->sp[SP_TP];
    int N = S->P.ncell;
    double dx = S->dx;
    double c = sqrt(2.0 * O_KB * S->P.Tg / O_MAR);
    double mu = O_MAL + O_MAR;
    int64_t alive = 0;
    for (int64_t k = 0; k < p->n; k++) {
        for (int64_t ev = 0; ev < max_events && p->alive[k]; ev++) {
            uint32_t e = p->nev[k];
            double v[3] = {p->vx[k], p->vy[k], p->vz[k]};
            double vm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            double nu, alpha = 1.0, va = 0.0, ma = 0.0;
            if (S->P.tp_model == 0) {
                nu = S->ngas * S->P.sigma_tp * orc_mean_rel_speed(vm, c);
            } else {
                /* VHS / M1: sigma(g) g = K g^alpha; candidates at the majorant rate
                 * n K (|v|^alpha + <|w|^alpha>) >= n K <|v - w|^alpha> (alpha <= 1) */
                alpha = 2.0 - 2.0 * S->P.omega;
                va = pow(vm, alpha);
                ma = pow(c, alpha) * tgamma(0.5 * (3.0 + alpha)) / tgamma(1.5);
                nu = S->ngas * orc_tp_sigma(S, 1.0) * (va + ma);
            }
            uint32_t f[4];
            draw(S->P.seed, p->id[k], e, PUR_TPF_FLIGHT, f);
            double tau = nu > 0.0 ? -log(u23(f[0])) / nu : INFINITY;
            if (!(tau < INFINITY) && v[0] == 0.0) break;       /* no gas, no motion across the gap */
            double xi0 = p->xi[k];
            double xi1 = xi0 + v[0] * tau / dx;
            if (xi1 <= 0.0 || xi1 >= (double)N) {            /* sticks at a wall */
                int el = xi1 <= 0.0 ? 0 : 1;
                double xw = el == 0 ? 0.0 : (double)N;
                tpf_segment(S, xi0, xw, v[0], (xw - xi0) * dx / v[0]);
                double E = 0.5 * O_MAL * vm * vm / O_QE;
                double ct = vm > 0.0 ? fabs(v[0]) / vm : 1.0;
                if (ct > 1.0) ct = 1.0;
                hist_add(S->sp_e[el], NB_SPE, E, 300.0);
                S->sp_ang[el][ang_bin(acos(ct) * 180.0 / O_PI)]++;
                S->cnt[el == 0 ? C_TPDEP_L : C_TPDEP_R]++;
                p->alive[k] = 0;
                p->xi[k] = xw;
                break;
            }
            tpf_segment(S, xi0, xi1, v[0], tau);
            p->xi[k] = xi1;
            double w[3];
            if (S->P.tp_model == 0) {
                orc_tpf_partner(S->P.seed, p->id[k], e, S->P.Tg, v, w);
            } else {
                /* candidate partner from (|v|^alpha + |w|^alpha) f(w): a Maxwellian with
                 * probability |v|^alpha / (|v|^alpha + <|w|^alpha>), else |w|^2/c^2 ~
                 * Gamma((3 + alpha)/2) with an isotropic direction; a real collision
                 * with probability |v - w|^alpha / (|v|^alpha + |w|^alpha), else none */
                uint32_t a[4], b[4];
                draw(S->P.seed, p->id[k], e, PUR_TPF_CAND, a);
                draw(S->P.seed, p->id[k], e, PUR_TPF_CAND + 1, b);
                if ((float)u23(a[0]) * ((float)va + (float)ma) < (float)va) {   /* in FP32 */
                    double vg = c / sqrt(2.0), n1, n2, n3, n4;
                    box_muller(a[1], a[2], &n1, &n2);
                    box_muller(a[3], b[0], &n3, &n4);
                    w[0] = vg * n1; w[1] = vg * n2; w[2] = vg * n3;
                } else {
                    double sp = c * sqrt(gamma_mt(0.5 * (3.0 + alpha), S->P.seed, p->id[k], e, PUR_TPF_GAMMA));
                    double dd[3];
                    iso_dir(a[3], b[0], dd);
                    w[0] = sp * dd[0]; w[1] = sp * dd[1]; w[2] = sp * dd[2];
                }
                double gg[3] = {v[0] - w[0], v[1] - w[1], v[2] - w[2]};
                double gmm = sqrt(gg[0] * gg[0] + gg[1] * gg[1] + gg[2] * gg[2]);
                double wm = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
                if (!((float)u23(b[1]) * ((float)va + (float)pow(wm, alpha)) < (float)pow(gmm, alpha))) {   /* FP32 */
                    p->nev[k] = e + 1u;                   /* a null event: the flight goes on */
                    continue;
                }
            }
            double g[3] = {v[0] - w[0], v[1] - w[1], v[2] - w[2]};
            double gm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
            uint32_t sc[4];
            draw(S->P.seed, p->id[k], e, PUR_TPF_SCATTER, sc);
            double d[3];
            orc_tp_scatter(S->P.tp_model, g, sc[0], sc[1], d);
            for (int i = 0; i < 3; i++) v[i] = (O_MAL * v[i] + O_MAR * w[i]) / mu + (O_MAR / mu) * gm * d[i];
            p->vx[k] = v[0]; p->vy[k] = v[1]; p->vz[k] = v[2];
            p->nev[k] = e + 1u;
            S->cnt[C_TPCOLL]++;
        }
        if (p->alive[k]) alive++;
    }
    return alive;
}

/* ======================= hypothesis checks =============================== */
int64_t orc_diag(const orc_state *S, int kind, double *out, int64_t cap);
/* Sec. "Hypotheses validation": (A) ions strike the electrodes nearly
 * mono-energetically and along the normal -- the width-to-peak ratio
 * dE/E_max of the ion energy distribution and the angular spread of the
 * impacts; (B) the charged and sputtered species are traces in the gas --
 * the largest n_Ar+/n_Ar and n_Al/n_Ar.  Readings: E_max is the centre of
 * the fullest bin, dE the full width at half maximum around it (the run of
 * bins from the peak whose counts stay at or above half the peak, edge to
 * edge); the spread is the root mean square impact angle over the angle
 * histogram (bin centres). */
double orc_width_to_peak(const double *h, int nb, double emax)
{
    int pk = 0;
    for (int b = 1; b < nb; b++) if (h[b] > h[pk]) pk = b;
    if (!(h[pk] > 0.0)) return 0.0;
    int lo = pk, hi = pk;
    while (lo > 0 && h[lo - 1] >= 0.5 * h[pk]) lo--;
    while (hi < nb - 1 && h[hi + 1] >= 0.5 * h[pk]) hi++;
    double bw = emax / nb;
    return (double)(hi - lo + 1) * bw / ((pk + 0.5) * bw);
}

double orc_rms_angle(const double *h, int nb)
{
    double s = 0.0, s2 = 0.0;
    for (int b = 0; b < nb; b++) {
        double th = b + 0.5;
        s += h[b];
        s2 += h[b] * th * th;
    }
    return s > 0.0 ? sqrt(s2 / s) : 0.0;
}

/* out: dE/E_max at x = 0 and x = L, rms impact angle (deg) at x = 0 and
 * x = L, max n_Ar+/n_Ar, max n_Al/n_Ar (time averages of the run so far) */
void orc_hypotheses(const orc_state *S, double out[6])
{
    int N = S->P.ncell;
    double *buf = (double *)malloc(sizeof(double) * (NB_IEADF_E * NB_ANG + N + 1));
    for (int el = 0; el < 2; el++) {
        orc_diag(S, 6 + el, buf, NB_IEDF);
        out[el] = orc_width_to_peak(buf, NB_IEDF, S->P.V0 > 0.0 ? 2.0 * S->P.V0 : 1.0);
        orc_diag(S, 8 + el, buf, NB_IEADF_E * NB_ANG);
        double ang[NB_ANG];
        for (int b = 0; b < NB_ANG; b++) ang[b] = 0.0;
        for (int e = 0; e < NB_IEADF_E; e++)
            for (int b = 0; b < NB_ANG; b++) ang[b] += buf[e * NB_ANG + b];
        out[2 + el] = orc_rms_angle(ang, NB_ANG);
    }
    double mi = 0.0, ma = 0.0;
    orc_diag(S, 2, buf, N + 1);
    for (int m = 0; m <= N; m++) mi = fmax(mi, buf[m]);
    orc_diag(S, 14, buf, N + 1);
    for (int m = 0; m <= N; m++) ma = fmax(ma, buf[m]);
    out[4] = mi / S->ngas;
    out[5] = ma / S->ngas;
    free(buf);
}

/* Mono-energetic source: n atoms launched from the left electrode with a
 * Thompson energy (cut off at Lambda E_ion) and a cosine angle; ids
 * tag | (atoms launched before + k). */
void orc_tp_launch_ids(orc_state *S, int64_t n, double E_ion, int64_t id0);
void orc_tp_launch(orc_state *S, int64_t n, double E_ion)
{
    int64_t id0 = S->tp_launched;
    S->tp_launched += n;
    orc_tp_launch_ids(S, n, E_ion, id0);
}

/* the atoms id0 .. id0 + n - 1 of a source (the share of one rank when a
 * source is split over several) */
void orc_tp_launch_ids(orc_state *S, int64_t n, double E_ion, int64_t id0)
{
    double Emax = lambda_ar_al() * E_ion;
    double N = (double)S->P.ncell;
    for (int64_t k = 0; k < n; k++) {
        uint64_t id = TAG[SP_TP] | (uint64_t)(id0 + k);
        uint32_t ce[4];
        draw(S->P.seed, id, 0, PUR_TP_LAUNCH, ce);
        double v[3];
        orc_emit(u23(ce[0]), u23(ce[1]), u23(ce[2]), Emax, 1.0, v);
        append(S, SP_TP, N * 0x1p-32, v[0], v[1], v[2], id, 0);
    }
}

/* ======================= diagnostics export ============================== */
/* kind: 0 phi, 1 n_e, 2 n_i (m^-3), 3 Gamma_e, 4 Gamma_i (m^-2 s^-1),
 * 5 EEDF, 6 IEDF left, 7 IEDF right, 8 IEADF left, 9 IEADF right,
 * 10 sputtered energy left, 11 right, 12 sputtered angle left, 13 right,
 * 14 TP density (m^-3), 15 TP mean v_x sum (m^-2 s^-1 like Gamma),
 * 16 event-driven TP residence time per cell (s), 17 its mean v_x per cell
 * (signed path over residence time, m/s; 0 where no time was spent).
 * Returns the number of values written. */
int64_t orc_diag(const orc_state *S, int kind, double *out, int64_t cap)
{
    int N = S->P.ncell;
    double dx = S->dx, w = S->P.w;
    int64_t n = 0;
#define PUT(v) do { if (n < cap) out[n] = (v); n++; } while (0)
    switch (kind) {
    case 0:
        for (int m = 0; m <= N; m++) PUT(S->n_avg ? S->sum_phi[m] / S->n_avg : 0.0);
        break;
    case 1: case 2:
        for (int m = 0; m <= N; m++) {
            double vol = (m == 0 || m == N) ? 0.5 * dx : dx;
            PUT(S->n_avg ? w * S->sum_q[kind - 1][m] / (4294967296.0 * vol * S->n_avg) : 0.0);
        }
        break;
    case 3: case 4:
        for (int m = 0; m <= N; m++) {
            double vol = (m == 0 || m == N) ? 0.5 * dx : dx;
            PUT(S->n_flux ? w * S->sum_flux[kind - 3][m] / (vol * S->n_flux) : 0.0);
        }
        break;
    case 5: for (int b = 0; b < NB_EEDF; b++) PUT((double)S->eedf[b]); break;
    case 6: case 7: for (int b = 0; b < NB_IEDF; b++) PUT((double)S->iedf[kind - 6][b]); break;
    case 8: case 9:
        for (int b = 0; b < NB_IEADF_E * NB_ANG; b++) PUT((double)S->ieadf[kind - 8][b]);
        break;
    case 10: case 11: for (int b = 0; b < NB_SPE; b++) PUT((double)S->sp_e[kind - 10][b]); break;
    case 12: case 13: for (int b = 0; b < NB_ANG; b++) PUT((double)S->sp_ang[kind - 12][b]); break;
    case 14: case 15:
        for (int m = 0; m <= N; m++) {
            double vol = (m == 0 || m == N) ? 0.5 * dx : dx;
            const double *a = kind == 14 ? S->tp_dens : S->tp_vx;
            PUT(S->n_tp_samp ? w * a[m] / (vol * S->n_tp_samp) : 0.0);
        }
        break;
    case 16: for (int j = 0; j < N; j++) PUT(S->tpf_time[j]); break;
    case 17:
        for (int j = 0; j < N; j++) PUT(S->tpf_time[j] > 0.0 ? S->tpf_disp[j] / S->tpf_time[j] : 0.0);
        break;
    default: break;
    }
#undef PUT
    return n;
}

void orc_reset_averages(orc_state *S)
{
    int N = S->P.ncell;
    for (int m = 0; m <= N; m++) {
        S->sum_q[0][m] = S->sum_q[1][m] = S->sum_phi[m] = 0.0;
        S->sum_flux[0][m] = S->sum_flux[1][m] = 0.0;
        S->tp_dens[m] = S->tp_vx[m] = 0.0;
    }
    S->n_avg = S->n_flux = S->n_tp_samp = 0;
    memset(S->eedf, 0, sizeof(int64_t) * NB_EEDF);
    for (int s = 0; s < 2; s++) {
        memset(S->iedf[s], 0, sizeof(int64_t) * NB_IEDF);
        memset(S->ieadf[s], 0, sizeof(int64_t) * NB_IEADF_E * NB_ANG);
        memset(S->sp_e[s], 0, sizeof(int64_t) * NB_SPE);
        memset(S->sp_ang[s], 0, sizeof(int64_t) * NB_ANG);
    }
}

uint32_t orc_get_step(const orc_state *S) { return S->step; }
void orc_set_step(orc_state *S, uint32_t l) { S->step = l; }
uint32_t orc_get_tp_step(const orc_state *S) { return S->tp_step; }
