// common.cuh -- device-side building blocks shared by the kernels of the
// GB300 PIC/MCC + test-particle engine (sm_103a).
//
// Everything here is written from arXiv:1607.04069 (Trieschmann, Schmidt &
// Mussenbrock) and from Salmon et al., SC'11 (Philox).  The random-stream
// layout (counter words, purpose codes, which word feeds which draw) is the
// engine's stream definition; it is fixed so that any implementation of the
// method that follows it draws the same numbers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pg {

// ---------------------------------------------------------------- constants
// CODATA 2018
constexpr double kQE = 1.602176634e-19;
constexpr double kME = 9.1093837015e-31;
constexpr double kAMU = 1.66053906660e-27;
constexpr double kKB = 1.380649e-23;
constexpr double kEPS0 = 8.8541878128e-12;
constexpr double kPI = 3.14159265358979323846;
constexpr double kMAR = 39.948 * kAMU;
constexpr double kMAL = 26.98 * kAMU;

// analytic cross sections (e-Ar: constant elastic; linear-onset excitation;
// one-term Lotz ionisation.  Ar+-Ar: 5e-19 (1 eV/eps)^1/2 per channel)
constexpr double kSigEl = 1e-19;
constexpr double kExcTh = 11.5;
constexpr double kExcSig = 1e-20;
constexpr double kIonTh = 15.8;
constexpr double kLotzA = 4.5e-18;
constexpr double kLotzQ = 6.0;
constexpr double kArpSig = 5e-19;
// sputtering of Al by Ar+: threshold, surface binding energy, max trials
constexpr double kSpTh = 30.0;
constexpr double kUb = 3.4;
constexpr int kSpMaxN = 16;

// histogram shapes
constexpr int kNbIedf = 512;     // ion energy, [0, 2 V0]
constexpr int kNbIeadfE = 128;   // ion energy x angle, energy axis
constexpr int kNbAng = 90;       // 1-degree bins, [0, 90)
constexpr int kNbEedf = 256;     // 0.25 eV bins, [0, 64)
constexpr int kNbSpE = 600;      // 0.5 eV bins, [0, 300)

// random-stream purposes (fourth counter word)
enum : uint32_t {
    kPurInit = 1, kPurColl = 2, kPurIonize = 3, kPurNewIon = 4, kPurBirthId = 5, kPurGas = 6,
    kPurGap = 7, kPurGap0 = 8,
    kPurSpTrial = 16, kPurSpEmit = 32, kPurSpId = 48, kPurTpGas = 64, kPurTpColl = 65,
    kPurTpLaunch = 66, kPurTpfFlight = 70, kPurTpfScatter = 71, kPurTpfPartner = 72, kPurTpfCand = 200,
    kPurTpfGamma = 202, kPurTpCand = 256, kPurTpGamma = 258, kPurTpGap = 290, kPurTpGap0 = 291
};

// species and id tags
enum { kE = 0, kI = 1, kTP = 2 };
__host__ __device__ constexpr uint64_t id_tag(int s) { return (uint64_t)s << 62; }
constexpr uint64_t kIdMask = (1ull << 62) - 1;

// counters (device, unsigned long long)
enum {
    kCntImpEL, kCntImpER, kCntImpIL, kCntImpIR, kCntIoniz, kCntSputL, kCntSputR, kCntTpDepL,
    kCntTpDepR, kCntNumerics, kCntElastic, kCntExcit, kCntCx, kCntIso, kCntTpColl, kCntCapacity,
    kNumCnt
};

// error bits of Ctl::err
enum : uint32_t { kErrCapacity = 1u, kErrNumerics = 2u, kErrIndex = 4u, kErrTimeout = 8u };

// ---------------------------------------------------------------- state
struct SpBuf {                 // one species, one ping-pong half (structure of arrays)
    void* pos;                 // uint32 fixed point x 2^32/L, or double x/dx (64-bit mode)
    float* vx;
    float* vy;
    float* vz;
    uint64_t* id;
    uint32_t* nev;             // step of the next null-collision candidate (e-, Ar+ only)
};

struct Ctl {                   // device control block
    long long n[3];            // slots in use per species (alive + removed holes)
    long long cap[3];
    unsigned int step, tp_step;
    unsigned int cur[3];       // active ping-pong half per species
    unsigned int field_override;   // next step uses E32 as given instead of solving
    long long n_avg, n_flux, n_tp_samp;
    long long sort_total;
    double sum_v;              // sum of the electrode voltage over the averaged steps
    long long wall_dn;         // ions minus electrons absorbed at x = 0 since creation (to the
                               // end of the last step launch; the series-capacitor circuit)
    // words updated by atomics while kernels run, each group on its own
    // 128-byte line so that their queues at L2 do not delay the others
    alignas(128) long long births[3];      // appended by the running kernel
    alignas(128) unsigned int done, tp_done, sort_done;
    alignas(128) unsigned int err;
    long long wall_delta;      // the running launch's share of wall_dn (moved over at commit)
    alignas(128) unsigned long long cnt[kNumCnt];   // counts of the TP kernels
    alignas(128) unsigned long long tpf_alive;      // atoms alive after an event-driven flight launch
};

// per-CTA event counts of the step launch: row b of Dev::tally belongs to
// CTA b, which adds its counts with reductions to its own row
constexpr int kMaxTallyRows = 4096;

// Time-averaged diagnostics are integer sums, so they are exact and
// independent of the order in which CTAs deposit.  Each node keeps two
// 64-bit words: the sum of the low 32 bits and the sum of the high 32 bits
// (arithmetic shift for signed moments) of the per-step value, so every step
// adds with fire-and-forget reductions and the total is hi 2^32 + lo.  The
// averaged potential follows from the averaged charge and electrode voltage,
// since the field solve is linear.
struct Diag {
    unsigned long long* sum_q[2];   // [2 (N+1)] per step: q_e, q_i (2^-32 particles)
    long long* sum_flux[2];         // [2 (N+1)] per sample: sum_k W_m(x_k) rint(v_x,k), 2^-16
    unsigned long long* tp_dens;    // [2 (N+1)] per TP sample: TP deposit
    long long* tp_vx;               // [2 (N+1)] per TP sample: TP v_x moment
    unsigned long long* iedf[2];
    unsigned long long* ieadf[2];
    unsigned long long* eedf;
    unsigned long long* sp_e[2];
    unsigned long long* sp_ang[2];
    // event-driven TP flight, per cell: residence time (2^-40 s) and signed
    // path (2^-32 L), each as a partial-cell term [N] plus a difference
    // array [N+1] of the cells crossed whole (value of cell j: part[j] +
    // sum_{i <= j} diff[i])
    long long *tpf_tpart, *tpf_tdiff, *tpf_dpart, *tpf_ddiff;
};

// Per-launch inputs of a step computed on the host: the electrode voltage of
// the step and 2 V / A split into an integer and a fraction, which keep the
// per-CTA field solve free of FP64 arithmetic.
struct StepArgs {
    double v_left;
    long long va_i;        // llrint(2 v_left / A)
    float va_f;            // 2 v_left / A - va_i
    float e_uniform;       // v_left / L, used when A == 0
    int field_mode;        // 0: integer path, 1: FP64 path (|2V/A| >= 2^62), 2: no space charge,
                           // 3: series capacitor (v_left is the source voltage; see Dev::circ_a)
    int accumulate;        // add the state of this step to the time averages
    unsigned int step;     // step index l (equal to Ctl::step)
    unsigned int cur[3];   // active ping-pong halves (equal to Ctl::cur)
};
enum { kFieldInt = 0, kFieldF64 = 1, kFieldUniform = 2, kFieldCircuit = 3 };

struct Dev {                   // everything a kernel needs, passed by value
    SpBuf buf[3][2];
    Ctl* ctl;
    Diag diag;
    // per-step charge and flux histograms, rotating over three slots: the
    // launch for step l solves from slot l%3, deposits x^{l+1} into slot
    // (l+1)%3 and clears slot (l+2)%3
    unsigned long long* qbuf[3][2];
    long long* fbuf[3][2];
    unsigned long long* tp_q;        // per-TP-step density histogram
    long long* tp_flux;              // per-TP-step v_x histogram
    float* E32;                      // field given by pic_set_field (override)
    double* E64;                     // FP64 field and potential of the current state
    double* phi;
    unsigned char* evflag[2];        // per-slot event flags, used when a CTA's event queue is full
    unsigned int* sort_cnt;          // [ncell] cell counts (sort scratch)
    unsigned int* sort_off;          // [ncell] running offsets (sort scratch)
    // geometry
    int ncell, kshift, pos64, pad0;
    double L, dx, inv_dx;
    // field solve: phi[m+1] - 2 phi[m] + phi[m-1] = -A q_net[m]; A = dx e w / (2^32 eps0)
    double A, V0, omega, dt, f_rf;
    // series blocking capacitor: the electrode potential in units of A/2 is
    //   2 phi_0 / A = circ_a V + circ_b (T_N + N q_0 + N 2^32 dn)
    // with T_N = sum_j (N - j) q_j over the deposit, dn the ions minus the
    // electrons absorbed at x = 0 (Ctl::wall_dn), circ_a = 2 (1 - beta) / A,
    // circ_b = 2 beta, beta = 1 / (1 + L c / eps0)
    double circ_a, circ_b;
    int circuit;
    int tp_mode;                     // TP step collisions: 0 thinned candidates, 1 the literal test
    // event-driven TP flight
    float tpf_c;                     // most probable speed of the gas, sqrt(2 k T / M_Ar)
    float tpf_nsig;                  // n sigma_tp, 1/m
    float tpf_scale;                 // 2^32 / L: fixed-point units per metre
    float tpf_kt;                    // 256 L: residence time (2^-40 s) per fixed-point unit at 1 m/s
    // TP collision model: 0 hard spheres (tp_nsig_dt, tpf_nsig); 1 VHS, 2 M1 with
    // sigma(g) g = K g^alpha
    int tp_model;
    float tp_alpha;                  // 2 - 2 omega
    float tp_nK_dt;                  // n K dt of tp_step (per-step rate n K g^alpha dt)
    float tpf_nK;                    // n K of the flight
    float tpf_malpha;                // <|w|^alpha> of the Maxwellian gas
    float tpf_gk;                    // (3 + alpha) / 2, the gamma shape of |w|^2/c^2
    // tabulated e-Ar cross sections (elastic, excitation, ionisation): (eV, m^2)
    // points, linear between them, constant beyond; xs_n 0: the analytic form
    const float2* xs_tab[3];
    int xs_n[3], xs_pad;
    float c2f;                       // A / (2 dx): E per unit of the integer bracket
    float tp_ma;                     // <|w|^alpha> of the gas (hard spheres: <|w|> = 2 c / sqrt(pi))
    unsigned int tp_wait_spin;       // polls of a TP tile's barrier before the wait gives up
    int tp_wait_test;                // 1: warp 0 of CTA 0 issues no copies, so its first wait runs out
    // push
    float qm_dt[2];                  // (q/m) dt
    float push32;                    // dt 2^32 / L  (fixed-point displacement per m/s)
    float pad1;
    double push64;                   // dt / dx      (cell-unit displacement per m/s)
    // collisions
    long long cap[3];                // slot capacities (as Ctl::cap)
    unsigned long long* tally;       // [kMaxTallyRows][kNumCnt] per-CTA event counts of the step launch
    double lam[2];                   // nu_max dt: candidate gaps are geometric with P_max = 1 - exp(-lam)
    float lamf[2];                   // the same rounded to float
    float ngas_f, nu_max_e, nu_max_i, eps_max;
    float vth_gas;                   // sqrt(k Tg / M_Ar)
    float tp_scale;                  // dt_tp 2^32 / L
    float tp_nsig_dt;                // n sigma_tp dt_tp
    float Emax_hist;                 // 2 V0 (ion histograms)
    int sputter, diag_every;
    unsigned int eedf_lo, eedf_hi;   // fixed-point window of the EEDF sample (0.45 L, 0.55 L)
    double eedf_lo64, eedf_hi64;
    uint64_t seed;
    unsigned long long* trace;       // optional per-CTA phase timestamps of the last step launch
};

// One discharge of a batched step launch (several independent discharges,
// one kernel per step): its descriptor, the step arguments of its RF phases,
// and the CTAs of the launch that work on it.
struct BatchEntry {
    Dev d;
    const StepArgs* phase;     // [period]: step l uses phase[l % period] (step, cur, accumulate set on device)
    unsigned int period;
    unsigned int acc_from;     // steps l >= acc_from enter the time averages
    int cta0, ncta;            // CTAs [cta0, cta0 + ncta) of the launch
};

// A chunk of the batched launch with resident CTAs: CTA slots [v0, v1) of
// discharge `member`, run one after another by one CTA.
struct BatchChunk {
    int member, v0, v1, pad;
};

// global nanosecond timer, comparable across SMs
__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// trace words per CTA: start, q loaded, field solved, prologue done, stream done, events done,
// flush done, end, species, events count | node range << 32, set-up done, copies issued,
// longest event (ns << 8 | kind), ionisations, tile flush (ns), unused
constexpr int kTraceSlots = 16;

// add a per-step value to a split (lo, hi) sum with fire-and-forget reductions
__device__ __forceinline__ void red_split(unsigned long long* p, unsigned long long v)
{
    atomicAdd(p, v & 0xffffffffull);
    if (v >> 32) atomicAdd(p + 1, v >> 32);
}
__device__ __forceinline__ void red_split_signed(long long* p, long long v)
{
    if (v & 0xffffffffll) atomicAdd((unsigned long long*)p, (unsigned long long)(v & 0xffffffffll));
    if (v >> 32) atomicAdd((unsigned long long*)(p + 1), (unsigned long long)(v >> 32));
}

// ---------------------------------------------------------------- Philox4x32-10
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const unsigned long long p0 = 0xD2511F53ull * c.x;     // one 32x32->64 product each
        const unsigned long long p1 = 0xCD9E8D57ull * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1,
                       (uint32_t)p0);
    }
    return c;
}

// N independent Philox4x32-10 blocks under one key, round by round, so their
// multiply chains overlap
template <int N>
__device__ __forceinline__ void philox_n(uint4 (&c)[N], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
#pragma unroll
        for (int u = 0; u < N; ++u) {
            const unsigned long long p0 = 0xD2511F53ull * c[u].x;
            const unsigned long long p1 = 0xCD9E8D57ull * c[u].z;
            c[u] = make_uint4((uint32_t)(p1 >> 32) ^ c[u].y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c[u].w ^ k1,
                              (uint32_t)p0);
        }
    }
}

__device__ __forceinline__ uint4 draw(uint64_t seed, uint64_t id, uint32_t step, uint32_t purpose)
{
    return philox(make_uint4((uint32_t)id, (uint32_t)(id >> 32), step, purpose), (uint32_t)seed,
                  (uint32_t)(seed >> 32));
}

// uniform in (0,1) on the 2^-23 grid (top 23 bits + 1/2), exact in float
__device__ __forceinline__ float u23(uint32_t w) { return ((float)(w >> 9) + 0.5f) * 0x1p-23f; }

// Steps from one null-collision candidate to the next (Sec. "Particle
// Collisions": every step is a candidate with P_max = 1 - exp(-nu_max dt),
// independently of the other steps): the free flight time tau = -ln R / nu_max
// (Sec. "Kinetic Particle Simulation") counted in steps and rounded up,
// gap = 1 + floor(-ln R / (nu_max dt)), whose law is geometric with P_max.
// The floor is that of the FP64 quotient, with R on the same 2^-23 grid as
// every other uniform.  FP64 is slow on this part, so the quotient is first
// formed in FP32 (logf within 1 ulp, lam rounded to float, one division:
// relative error below 3e-7); when no integer lies within 4e-7 x of the FP32
// value, its floor is the floor of the FP64 quotient, and only the other
// cases evaluate the FP64 expression.
__device__ __forceinline__ bool gap_fast(float lamf, uint32_t w, uint32_t& gap)
{
    const float uf = ((float)(w >> 9) + 0.5f) * 0x1p-23f;      // exact in float (24 bits)
    const float xf = -logf(uf) / lamf;
    if (!(xf < 1.0e6f)) return false;
    const float dl = 4e-7f * xf + 1e-6f;
    const float a = floorf(xf - dl), b = floorf(xf + dl);
    if (a != b) return false;
    gap = 1u + (uint32_t)a;
    return true;
}
__device__ __forceinline__ uint32_t gap_exact(double lam, uint32_t w)
{
    const double u = ((double)(w >> 9) + 0.5) * 0x1p-23;
    const double x = -log(u) / lam;
    if (!(x < 2147483646.0)) return 2147483647u;
    return 1u + (uint32_t)floor(x);
}
__device__ __forceinline__ uint32_t gap_steps(double lam, float lamf, uint32_t w)
{
    uint32_t g;
    return gap_fast(lamf, w, g) ? g : gap_exact(lam, w);
}

// step of the first candidate of an e- or Ar+ that is first pushed at step l0
__device__ __forceinline__ uint32_t entry_nev(const Dev& d, int s, uint64_t id, uint32_t l0)
{
    return l0 - 1u + gap_steps(d.lam[s], d.lamf[s], draw(d.seed, id, l0, kPurGap0).x);
}

__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b)
{
    const float r = sqrtf(-2.0f * logf(u23(a)));
    float s, c;
    sincospif(2.0f * u23(b), &s, &c);
    return make_float2(r * c, r * s);
}

__device__ __forceinline__ float3 iso_dir(uint32_t a, uint32_t b)
{
    const float c = 1.0f - 2.0f * u23(a);
    const float s = sqrtf(fmaxf(0.0f, 1.0f - c * c));
    float sp, cp;
    sincospif(2.0f * u23(b), &sp, &cp);
    return make_float3(c, s * cp, s * sp);
}

__device__ __forceinline__ uint64_t child_id(uint32_t lo, uint32_t hi, int s)
{
    return ((((uint64_t)hi << 32) | lo) & kIdMask) | id_tag(s);
}

// Thompson energy (truncated at Emax, by inversion of (E/(E+Ub))^2) and cosine
// angle; dir = +1 into +x (left electrode), -1 into -x.
__device__ __forceinline__ float3 emit(float uE, float uT, float uP, float Emax, float dir)
{
    const float t = Emax / (Emax + (float)kUb);
    const float s = sqrtf(uE * t * t);
    const float Es = (float)kUb * s / (1.0f - s);
    const float speed = sqrtf(2.0f * Es * (float)(kQE / kMAL));
    const float ct = sqrtf(uT);
    const float st = sqrtf(fmaxf(0.0f, 1.0f - uT));
    float sp, cp;
    sincospif(2.0f * uP, &sp, &cp);
    return make_float3(dir * speed * ct, speed * st * cp, speed * st * sp);
}

__device__ __forceinline__ float lambda_ar_al()
{
    return (float)(4.0 * kMAR * kMAL / ((kMAR + kMAL) * (kMAR + kMAL)));
}

// ---------------------------------------------------------------- bulk copies (TMA)
// One-dimensional bulk copies global -> shared memory by the tensor memory
// accelerator, completing on a shared-memory mbarrier (transaction count in
// bytes).  Addresses and sizes are multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// make the barrier initialisation visible to the bulk-copy (async) proxy
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// order earlier generic-proxy accesses of shared memory before later bulk copies into it
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Wait for the barrier's phase `parity` to complete, at most max_tries polls
// (each may suspend the thread for a short while); false if it never did.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned max_tries)
{
    const unsigned a = smem_addr(bar);
    for (unsigned i = 0; i < max_tries; ++i) {
        unsigned ok;
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(ok)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (ok) return true;
    }
    return false;
}

// ---------------------------------------------------------------- histogram bins
// Bin of an already scaled value t (bin width 1) among nb bins: below the
// range the first bin, at or above it -- and NaN -- the last.  The value is
// clamped before the conversion, so no out-of-range float is converted.
__device__ __forceinline__ int clamp_bin(float t, int nb)
{
    if (!(t < (float)nb)) return nb - 1;
    if (!(t >= 0.0f)) return 0;
    return (int)t;
}
// bin of x on [0, xmax) in nb bins
__device__ __forceinline__ int hist_bin(float x, float xmax, int nb) { return clamp_bin(x / xmax * (float)nb, nb); }

// ---------------------------------------------------------------- warp deposit
// Linear weighting of one particle per lane into a shared int64 histogram:
// node j gets 2^32 - wr, node j+1 gets wr.  Lanes whose cells span at most
// 4 consecutive cells are summed in registers first (counts by ballot,
// weights by two 32-bit reductions of 24+8 bits), so a sorted warp issues a
// handful of atomics instead of 64.  Integer sums: exact, order-independent.
__device__ __forceinline__ void warp_deposit(unsigned long long* sq, bool act, uint32_t j, uint32_t wr)
{
    const unsigned FULL = 0xffffffffu;
    const uint32_t jmin = __reduce_min_sync(FULL, act ? j : 0xffffffffu);
    if (jmin == 0xffffffffu) return;
    const uint32_t jmax = __reduce_max_sync(FULL, act ? j : 0u);
    const int lane = threadIdx.x & 31;
    if (jmax - jmin < 4) {
        const int span = (int)(jmax - jmin);
        unsigned long long prevR = 0;
        for (int c = 0; c <= span; ++c) {
            const bool in = act && (j == jmin + (uint32_t)c);
            const unsigned m = __ballot_sync(FULL, in);
            const uint32_t hi = __reduce_add_sync(FULL, in ? (wr >> 8) : 0u);
            const uint32_t lo = __reduce_add_sync(FULL, in ? (wr & 0xffu) : 0u);
            const unsigned long long R = ((unsigned long long)hi << 8) + lo;
            const unsigned long long node = ((unsigned long long)__popc(m) << 32) - R + prevR;
            if (lane == c && node) atomicAdd(&sq[jmin + c], node);
            prevR = R;
        }
        if (lane == span + 1 && prevR) atomicAdd(&sq[jmin + span + 1], prevR);
    } else if (act) {
        atomicAdd(&sq[j], (1ull << 32) - wr);
        if (wr) atomicAdd(&sq[j + 1], (unsigned long long)wr);
    }
}

// cell index and right-node weight of a position
__device__ __forceinline__ void cell_of(uint32_t pos, int kshift, uint32_t& j, uint32_t& wr)
{
    j = pos >> (32 - kshift);
    wr = pos << kshift;            // (xi - j) 2^32, exact
}
__device__ __forceinline__ void cell_of(double xi, int, uint32_t& j, uint32_t& wr)
{
    const double fj = floor(xi);
    j = (uint32_t)fj;
    wr = (uint32_t)((xi - fj) * 4294967296.0);   // floor of f 2^32 (f 2^32 exact, f < 1)
}

__device__ __forceinline__ bool is_alive(uint32_t pos) { return pos != 0u; }
__device__ __forceinline__ bool is_alive(double xi) { return xi >= 0.0; }

}  // namespace pg
