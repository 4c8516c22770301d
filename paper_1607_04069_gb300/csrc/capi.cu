// capi.cu -- host side of the C ABI declared in include/pic_gb300.h.
//
// Owns the device state of one discharge (one allocation, carved into the
// structure-of-arrays particle store, the per-step histograms and the
// diagnostic accumulators), schedules the per-step kernels on the caller's
// stream and converts diagnostics to physical units on the host.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pic_gb300.h"
#include "common.cuh"
#include "launch.h"

using namespace pg;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PIC_ERR_OUT_OF_MEMORY : PIC_ERR_CUDA;
}

#define CK(expr)                                                         \
    do {                                                                 \
        cudaError_t e__ = (expr);                                        \
        if (e__ != cudaSuccess) return cuda_fail(e__, #expr);            \
    } while (0)

struct Timer {                       // CUDA-event pairs around launches
    std::vector<cudaEvent_t> ev;
    size_t used = 0;
    double ms = 0.0;
    long long launches = 0;
};

}  // namespace

// error detail set by the library's other translation units
void pg::set_last_error(const char* msg) { g_err = msg; }

struct pic_ctx {
    pic_params p;
    int device = 0;
    cudaStream_t stream = nullptr;
    Dev d;                           // kernel descriptor (device pointers + constants)
    Dev d_coupled;                   // same, with the coupled TP time step
    void* arena = nullptr;
    size_t arena_bytes = 0, small_bytes = 0;
    int sms = 0, grid_mover = 0, grid_tp = 0, grid_tp_sample = 0, grid_sort = 0;
    long long h_step = 0, h_tp_step = 0, tp_launched = 0;
    float tp_gap_scale = 0.0f;       // TP step length (as Dev::tp_scale) the kept candidate gaps belong to
    long long exch_stride = 0;       // words per array of a rotating deposit slot
    long long acc_upto = 0;          // last step whose state entered the time averages
    unsigned int cur[3] = {0, 0, 0}; // active ping-pong halves (each compaction flips one)
    long long period = 0;            // steps per RF period when that is a whole number, else 0
    double circ_beta = 0.0;          // series capacitor: 1 / (1 + L c / eps0)
    std::vector<double> xs_e[3], xs_s[3];   // tabulated e-Ar cross sections (eV, m^2), empty: analytic
    float2* xs_dev[3] = {nullptr, nullptr, nullptr};
    double derived[8];
    bool timing = false;
    Timer timers[3];
};

namespace {

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2(int v)
{
    int k = 0;
    while ((1 << k) < v) ++k;
    return k;
}

// Carve the arena.  Small, zero-initialised items first.
struct Layout {
    size_t off = 0;
    template <typename T>
    T* take(char* base, size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T* p = (T*)(base + off);
        off += count * sizeof(T);
        return p;
    }
};

void carve(pic_ctx* c, char* base, size_t* small_end, size_t* total)
{
    Layout L;
    const int N1 = c->p.n_cells + 1;
    Dev& d = c->d;
    d.ctl = L.take<Ctl>(base, 1);
    // each rotating slot is one block [q_e | q_i | f_e | f_i] of exch_stride words
    // per array (256-byte aligned), so that it can be summed over ranks in one call
    const size_t stride = ((size_t)N1 + 31) & ~(size_t)31;
    c->exch_stride = (long long)stride;
    for (int k = 0; k < 3; ++k) {
        unsigned long long* blk = L.take<unsigned long long>(base, 4 * stride);
        d.qbuf[k][0] = blk;
        d.qbuf[k][1] = blk + stride;
        d.fbuf[k][0] = (long long*)(blk + 2 * stride);
        d.fbuf[k][1] = (long long*)(blk + 3 * stride);
    }
    for (int s = 0; s < 2; ++s) {
        d.diag.sum_q[s] = L.take<unsigned long long>(base, 2 * N1);
        d.diag.sum_flux[s] = L.take<long long>(base, 2 * N1);
        d.diag.iedf[s] = L.take<unsigned long long>(base, kNbIedf);
        d.diag.ieadf[s] = L.take<unsigned long long>(base, kNbIeadfE * kNbAng);
        d.diag.sp_e[s] = L.take<unsigned long long>(base, kNbSpE);
        d.diag.sp_ang[s] = L.take<unsigned long long>(base, kNbAng);
    }
    d.diag.tp_dens = L.take<unsigned long long>(base, 2 * N1);
    d.diag.tpf_tpart = L.take<long long>(base, N1);
    d.diag.tpf_tdiff = L.take<long long>(base, N1);
    d.diag.tpf_dpart = L.take<long long>(base, N1);
    d.diag.tpf_ddiff = L.take<long long>(base, N1);
    d.diag.tp_vx = L.take<long long>(base, 2 * N1);
    d.diag.eedf = L.take<unsigned long long>(base, kNbEedf);
    d.tp_q = L.take<unsigned long long>(base, N1);
    d.tp_flux = L.take<long long>(base, N1);
    d.E32 = L.take<float>(base, N1);
    d.E64 = L.take<double>(base, N1);
    d.phi = L.take<double>(base, N1);
    d.sort_cnt = L.take<unsigned int>(base, c->p.n_cells);
    d.sort_off = L.take<unsigned int>(base, c->p.n_cells);
    d.tally = L.take<unsigned long long>(base, (size_t)kMaxTallyRows * kNumCnt);
    *small_end = (L.off + 255) & ~(size_t)255;
    const long long cap[3] = {c->p.cap_e, c->p.cap_i, c->p.cap_tp};
    for (int s = 0; s < 3; ++s)
        for (int h = 0; h < 2; ++h) {
            SpBuf& B = d.buf[s][h];
            const size_t n = (size_t)((cap[s] > 0 ? cap[s] : 1) + 3) & ~(size_t)3;   // whole 4-slot groups
            if (c->p.pos_precision == 64 && s != kTP) B.pos = L.take<double>(base, n);
            else B.pos = L.take<uint32_t>(base, n);
            B.vx = L.take<float>(base, n);
            B.vy = L.take<float>(base, n);
            B.vz = L.take<float>(base, n);
            B.id = L.take<uint64_t>(base, n);
            B.nev = L.take<uint32_t>(base, n);    // TP: index of the next flight event
        }
    for (int s = 0; s < 2; ++s) d.evflag[s] = L.take<unsigned char>(base, (size_t)(cap[s] > 0 ? cap[s] : 1) + 4);
    *total = (L.off + 255) & ~(size_t)255;
}

// capacities left at 0: the initial load plus a quarter plus 65536 slots
void default_caps(pic_params* q)
{
    if (q->cap_e == 0) q->cap_e = q->n_e0 + q->n_e0 / 4 + 65536;
    if (q->cap_i == 0) q->cap_i = q->n_i0 + q->n_i0 / 4 + 65536;
    if (q->cap_tp == 0) q->cap_tp = 65536;
}

int validate(const pic_params* p)
{
    if (!p) return fail(PIC_ERR_INVALID_ARG, "params is NULL");
    if (!(p->gap_m > 0) || !(p->dt > 0) || !(p->gas_temp_k > 0) || !(p->pressure_pa >= 0) ||
        !(p->weight >= 0) || !(p->rf_freq_hz >= 0))
        return fail(PIC_ERR_INVALID_ARG, "gap, dt and gas temperature must be > 0; pressure, weight, "
                                         "frequency >= 0");
    if (!pow2(p->n_cells) || p->n_cells < 4 || p->n_cells > 4096)
        return fail(PIC_ERR_INVALID_ARG, "n_cells must be a power of two in [4, 4096]");
    if (p->pos_precision != 32 && p->pos_precision != 64)
        return fail(PIC_ERR_INVALID_ARG, "pos_precision must be 32 or 64");
    if (p->id_offset < 0 || p->id_offset + (p->n_e0 > p->n_i0 ? p->n_e0 : p->n_i0) > (1ll << 61))
        return fail(PIC_ERR_INVALID_ARG, "id_offset must be >= 0 and leave the ids below 2^61");
    if (p->n_e0 < 0 || p->n_i0 < 0 || p->cap_e < p->n_e0 || p->cap_i < p->n_i0 || p->cap_tp < 0)
        return fail(PIC_ERR_INVALID_ARG, "counts must be >= 0 and within the capacities");
    if (p->cap_e >= (1ll << 31) || p->cap_i >= (1ll << 31) || p->cap_tp >= (1ll << 32) - 1)
        return fail(PIC_ERR_INVALID_ARG, "capacity above the 32-bit slot index range");
    if (p->tp_every < 0 || p->diag_every < 0 || p->sort_every_e < 0 || p->sort_every_i < 0 ||
        p->sort_every_tp < 0 || p->ctas_per_sm < 0)
        return fail(PIC_ERR_INVALID_ARG, "negative period");
    if (!(p->tp_dt >= 0) || !(p->sigma_tp >= 0)) return fail(PIC_ERR_INVALID_ARG, "tp_dt, sigma_tp >= 0");
    if (p->tp_mode != 0 && p->tp_mode != 1) return fail(PIC_ERR_INVALID_ARG, "tp_mode must be 0 or 1");
    if (p->tp_model < 0 || p->tp_model > 2 ||
        (p->tp_model > 0 && !(p->tp_dref > 0 && p->tp_omega >= 0.5 && p->tp_omega <= 1.0 && p->tp_tref > 0)))
        return fail(PIC_ERR_INVALID_ARG, "tp_model 0..2; VHS/M1 need tp_dref > 0, 0.5 <= tp_omega <= 1, tp_tref > 0");
    if ((p->waveform != 0 && p->waveform != 1) || (p->circuit != 0 && p->circuit != 1))
        return fail(PIC_ERR_INVALID_ARG, "waveform and circuit must be 0 or 1");
    if (!std::isfinite(p->rf_phase) || (p->circuit == 1 && !(p->c_block >= 0)))
        return fail(PIC_ERR_INVALID_ARG, "rf_phase must be finite and c_block >= 0");
    return PIC_OK;
}

// Null-collision bounds (Sec. "Particle Collisions"): nu_max = max over energy
// of n sigma_sum(eps) sqrt(2 eps/m_r).  Electrons: sum of the closed-form
// maxima of the three cross sections at the highest admitted energy
// eps_max = 2 V0 + 100 eV.  Ar+: sigma(eps) g is constant, nu_max exact.
void derive(pic_ctx* c)
{
    const pic_params& p = c->p;
    const double ngas = p.pressure_pa / (kKB * p.gas_temp_k);
    const double dx = p.gap_m / (double)p.n_cells;
    // null-collision energy bound: twice the peak source voltage (V0 for the
    // sine, 2 V0 for the two-harmonic waveform) plus 100 eV
    const double eps_max = 2.0 * (p.waveform == 1 ? 2.0 * p.rf_volt_v : p.rf_volt_v) + 100.0;
    // closed-form maxima of the analytic cross sections; a tabulated process
    // contributes its largest tabulated value
    double sig_max[3] = {kSigEl, kExcSig, kLotzA * kLotzQ / (std::exp(1.0) * kIonTh * kIonTh)};
    for (int q = 0; q < 3; ++q)
        if (!c->xs_s[q].empty()) sig_max[q] = *std::max_element(c->xs_s[q].begin(), c->xs_s[q].end());
    const double sig_sum_max = sig_max[0] + sig_max[1] + sig_max[2];
    const double nu_max_e = ngas * sig_sum_max * std::sqrt(2.0 * eps_max * kQE / kME);
    const double mr = kMAR / 2.0;
    const double nu_max_i = 2.0 * ngas * kArpSig * std::sqrt(2.0 * kQE / mr);
    const double p_max_e = 1.0 - std::exp(-(nu_max_e * p.dt));
    const double p_max_i = 1.0 - std::exp(-(nu_max_i * p.dt));
    const double lam = 4.0 * kMAR * kMAL / ((kMAR + kMAL) * (kMAR + kMAL));
    double* o = c->derived;
    o[0] = ngas; o[1] = dx; o[2] = nu_max_e; o[3] = nu_max_i; o[4] = p_max_e; o[5] = p_max_i;
    o[6] = eps_max; o[7] = lam;

    Dev& d = c->d;
    d.ncell = p.n_cells;
    d.kshift = ilog2(p.n_cells);
    d.pos64 = p.pos_precision == 64;
    d.L = p.gap_m;
    d.dx = dx;
    d.inv_dx = 1.0 / dx;
    d.A = dx * kQE * p.weight / (4294967296.0 * kEPS0);
    d.c2f = (float)(0.5 * d.A / dx);
    d.V0 = p.rf_volt_v;
    d.omega = 2.0 * kPI * p.rf_freq_hz;
    d.f_rf = p.rf_freq_hz;
    d.dt = p.dt;
    d.qm_dt[kE] = (float)(-kQE / kME * p.dt);
    d.qm_dt[kI] = (float)(kQE / kMAR * p.dt);
    d.push32 = (float)(p.dt * 4294967296.0 / p.gap_m);
    d.push64 = p.dt / dx;
    d.cap[kE] = p.cap_e;
    d.cap[kI] = p.cap_i;
    d.cap[kTP] = p.cap_tp;
    // series blocking capacitor (an infinite one is the ideal source)
    d.circuit = p.circuit == 1 && std::isfinite(p.c_block);
    const double beta = d.circuit ? 1.0 / (1.0 + p.gap_m * p.c_block / kEPS0) : 0.0;
    c->circ_beta = beta;
    d.circ_a = d.A > 0.0 ? 2.0 * (1.0 - beta) / d.A : 0.0;
    d.circ_b = 2.0 * beta;
    c->period = 0;
    if (p.rf_freq_hz > 0) {
        const double per = 1.0 / (p.rf_freq_hz * p.dt);
        const long long P = std::llrint(per);
        if (P >= 1 && P <= (1ll << 24) && std::fabs((double)P * p.rf_freq_hz * p.dt - 1.0) < 1e-9) c->period = P;
    }
    d.lam[kE] = nu_max_e * p.dt;
    d.lam[kI] = nu_max_i * p.dt;
    d.lamf[kE] = (float)d.lam[kE];
    d.lamf[kI] = (float)d.lam[kI];
    d.ngas_f = (float)ngas;
    d.nu_max_e = (float)nu_max_e;
    d.nu_max_i = (float)nu_max_i;
    d.eps_max = (float)eps_max;
    d.vth_gas = (float)std::sqrt(kKB * p.gas_temp_k / kMAR);
    d.tp_scale = (float)(p.tp_dt * 4294967296.0 / p.gap_m);
    d.tp_nsig_dt = (float)(ngas * p.sigma_tp * p.tp_dt);
    d.tpf_c = (float)std::sqrt(2.0 * kKB * p.gas_temp_k / kMAR);
    d.tpf_nsig = (float)(ngas * p.sigma_tp);
    d.tpf_scale = (float)(4294967296.0 / p.gap_m);
    d.tpf_kt = (float)(256.0 * p.gap_m);
    d.tp_model = p.tp_model;
    d.tp_mode = p.tp_mode;
    d.tp_wait_spin = 1u << 22;                 // polls: far beyond any copy's latency
    d.tp_wait_test = 0;
    d.tp_ma = (float)(2.0 * std::sqrt(2.0 * kKB * p.gas_temp_k / kMAR) / std::sqrt(kPI));   // <|w|>
    double nK = 0.0;                                    // n K of the VHS / M1 law
    if (p.tp_model > 0) {
        // sigma(g) g = K g^alpha, K = pi d^2 (2 k T_ref / m_r)^(omega - 1/2) / Gamma(5/2 - omega)
        const double mr = kMAL * kMAR / (kMAL + kMAR);
        const double dd = p.tp_model == 2 ? std::sqrt(4.0 / 3.0) * p.tp_dref : p.tp_dref;
        const double K = kPI * dd * dd * std::pow(2.0 * kKB * p.tp_tref / mr, p.tp_omega - 0.5) /
                         std::tgamma(2.5 - p.tp_omega);
        const double alpha = 2.0 - 2.0 * p.tp_omega;
        const double c = std::sqrt(2.0 * kKB * p.gas_temp_k / kMAR);
        d.tp_alpha = (float)alpha;
        nK = ngas * K;
        d.tp_nK_dt = (float)(nK * p.tp_dt);
        d.tpf_nK = (float)nK;
        d.tpf_malpha = (float)(std::pow(c, alpha) * std::tgamma(0.5 * (3.0 + alpha)) / std::tgamma(1.5));
        d.tp_ma = d.tpf_malpha;
        d.tpf_gk = (float)(0.5 * (3.0 + alpha));
    }
    d.Emax_hist = (float)(2.0 * p.rf_volt_v > 0 ? 2.0 * p.rf_volt_v : 1.0);
    d.sputter = p.sputter_enable != 0;
    d.diag_every = p.diag_every;
    d.eedf_lo = (unsigned int)std::ceil(0.45 * 4294967296.0);
    d.eedf_hi = (unsigned int)std::ceil(0.55 * 4294967296.0);
    d.eedf_lo64 = 0.45 * p.n_cells;
    d.eedf_hi64 = 0.55 * p.n_cells;
    d.seed = p.seed;
    c->d_coupled = d;
    const double dtc = p.tp_every * p.dt;
    c->d_coupled.tp_scale = (float)(dtc * 4294967296.0 / p.gap_m);
    c->d_coupled.tp_nsig_dt = (float)(ngas * p.sigma_tp * dtc);
    c->d_coupled.tp_nK_dt = (float)(nK * dtc);
}

void sync_desc(pic_ctx* c)          // keep the coupled descriptor's pointers in step
{
    const Dev keep = c->d_coupled;
    c->d_coupled = c->d;
    c->d_coupled.tp_scale = keep.tp_scale;
    c->d_coupled.tp_nsig_dt = keep.tp_nsig_dt;
    c->d_coupled.tp_nK_dt = keep.tp_nK_dt;
}

// source voltage at step l (Sec. "Simulation Scenario"): V0 sin(w t), or the
// fundamental and its harmonic V0 [cos(w t + phase) + cos(2 w t)]; the phase
// of step l is taken at l mod period when the period is a whole number of steps
double v_left_at(const pic_ctx* c, long long l)
{
    const long long lp = c->period > 0 ? l % c->period : l;
    const double wt = 2.0 * kPI * c->p.rf_freq_hz * (double)lp * c->p.dt;
    if (c->p.waveform == 1) return c->p.rf_volt_v * (std::cos(wt + c->p.rf_phase) + std::cos(2.0 * wt));
    return c->p.rf_volt_v * std::sin(wt);
}

// the voltage the FP64 field solve starts from: the source voltage, or with
// the series capacitor and no space charge the divided one
double field_v_at(const pic_ctx* c, long long l)
{
    const double V = v_left_at(c, l);
    return c->d.circuit && c->d.A == 0.0 ? (1.0 - c->circ_beta) * V : V;
}

StepArgs step_args(const pic_ctx* c, long long l, int accumulate)
{
    StepArgs a;
    std::memset(&a, 0, sizeof a);
    a.v_left = v_left_at(c, l);
    a.accumulate = accumulate;
    a.step = (unsigned int)l;
    for (int s = 0; s < 3; ++s) a.cur[s] = c->cur[s];
    if (c->d.circuit) {
        if (c->d.A == 0.0) {                     // no space charge: the capacitive divider
            a.v_left *= 1.0 - c->circ_beta;
            a.field_mode = kFieldUniform;
            a.e_uniform = (float)(a.v_left / c->p.gap_m);
        } else {
            a.field_mode = kFieldCircuit;        // the launch forms the electrode potential
        }
        return a;
    }
    if (c->d.A == 0.0) {
        a.field_mode = kFieldUniform;
        a.e_uniform = (float)(a.v_left / c->p.gap_m);
    } else {
        const double va = 2.0 * a.v_left / c->d.A;
        if (std::fabs(va) < 4.0e18) {
            a.field_mode = kFieldInt;
            a.va_i = std::llrint(va);
            a.va_f = (float)(va - (double)a.va_i);
        } else {
            a.field_mode = kFieldF64;
        }
    }
    return a;
}

int timer_begin(pic_ctx* c, int k, cudaEvent_t* stop)
{
    *stop = nullptr;
    if (!c->timing) return PIC_OK;
    Timer& t = c->timers[k];
    if (t.used + 2 > t.ev.size()) {
        for (int i = 0; i < 64; ++i) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            t.ev.push_back(e);
        }
    }
    CK(cudaEventRecord(t.ev[t.used], c->stream));
    *stop = t.ev[t.used + 1];
    t.used += 2;
    return PIC_OK;
}

int timer_end(pic_ctx* c, cudaEvent_t stop)
{
    if (stop) CK(cudaEventRecord(stop, c->stream));
    return PIC_OK;
}

int timers_collect(pic_ctx* c)
{
    for (int k = 0; k < 3; ++k) {
        Timer& t = c->timers[k];
        for (size_t i = 0; i + 1 < t.used; i += 2) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, t.ev[i], t.ev[i + 1]));
            t.ms += ms;
            t.launches += 1;
        }
        t.used = 0;
    }
    return PIC_OK;
}

int run_tp_step(pic_ctx* c, const Dev& d)
{
    cudaEvent_t stop;
    int rc = timer_begin(c, 1, &stop);
    if (rc) return rc;
    if (d.tp_mode == 0 && d.tp_scale != c->tp_gap_scale) {
        // candidate gaps kept per atom were drawn for another TP step length:
        // every atom draws its next candidate afresh at this step (the
        // candidate process is memoryless)
        for (int h = 0; h < 2; ++h)
            CK(cudaMemsetAsync(d.buf[kTP][h].nev, 0, ((size_t)(c->p.cap_tp > 0 ? c->p.cap_tp : 1) + 3) / 4 * 16,
                               c->stream));
        c->tp_gap_scale = d.tp_scale;
    }
    // the device's TP step counter (ctl->tp_step) advances with every launch, as h_tp_step does
    const bool sample = d.diag_every > 0 && (c->h_tp_step + 1) % d.diag_every == 0;
    CK(launch_tp_step(d, sample ? c->grid_tp_sample : c->grid_tp, sample, c->stream));
    rc = timer_end(c, stop);
    if (rc) return rc;
    c->h_tp_step++;
    if (c->p.sort_every_tp > 0 && c->h_tp_step % c->p.sort_every_tp == 0) {
        rc = timer_begin(c, 2, &stop);
        if (rc) return rc;
        CK(launch_sort(c->d, kTP, c->grid_sort, c->stream));
        c->cur[kTP] ^= 1u;
        rc = timer_end(c, stop);
    }
    return rc;
}

}  // namespace

extern "C" {

int pic_params_default(pic_params* p)
{
    if (!p) return fail(PIC_ERR_INVALID_ARG, "p is NULL");
    std::memset(p, 0, sizeof(*p));
    p->gap_m = 0.025;
    p->pressure_pa = 3.0;
    p->gas_temp_k = 300.0;
    p->rf_freq_hz = 13.56e6;
    p->rf_volt_v = 100.0;
    p->n_e0 = p->n_i0 = 20000;
    p->weight = 1e15 * p->gap_m / 20000.0;
    p->dt = 1.0 / 13.56e6 / 400.0;
    p->te0_ev = 2.0;
    p->ti0_ev = 0.026;
    p->tp_dt = 1e-9;
    p->sigma_tp = 3e-19;
    p->seed = 1234;
    p->n_cells = 128;
    p->pos_precision = 64;
    p->diag_every = 10;
    p->sort_every_e = 20;
    p->sort_every_i = 200;
    p->sort_every_tp = 50;
    return PIC_OK;
}

double pic_vhs_dref(double mu_ref, double t_ref, double omega, double mass_kg)
{
    return std::sqrt(15.0 * std::sqrt(mass_kg * kKB * t_ref / kPI) / (8.0 * (2.5 - omega) * (3.5 - omega) * mu_ref));
}

int pic_state_bytes(const pic_params* pin, int64_t* bytes)
{
    if (!pin || !bytes) return fail(PIC_ERR_INVALID_ARG, "NULL argument");
    pic_params q = *pin;
    default_caps(&q);
    int rc = validate(&q);
    if (rc) return rc;
    pic_ctx tmp;
    tmp.p = q;
    derive(&tmp);
    size_t small_end = 0, total = 0;
    carve(&tmp, nullptr, &small_end, &total);
    *bytes = (int64_t)total;
    return PIC_OK;
}

int pic_create(const pic_params* pin, void* stream, pic_ctx** out)
{
    if (!out) return fail(PIC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!pin) return fail(PIC_ERR_INVALID_ARG, "params is NULL");
    pic_params q = *pin;
    default_caps(&q);
    int rc = validate(&q);
    if (rc) return rc;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(PIC_ERR_NO_DEVICE, "no CUDA device visible");
    pic_ctx* c = new pic_ctx();
    c->p = q;
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);
    derive(c);
    if (c->p.strict && c->p.n_e0 > 0) {
        const double n0 = c->p.weight * (double)c->p.n_e0 / c->p.gap_m;
        const double lam_d = std::sqrt(kEPS0 * c->p.te0_ev / (n0 * kQE));
        const double wp = std::sqrt(n0 * kQE * kQE / (kEPS0 * kME));
        if (!(c->d.dx < lam_d) || !(wp * c->p.dt < 1.0)) {
            char buf[160];
            std::snprintf(buf, sizeof buf, "dx = %.3g m vs lambda_D = %.3g m, w_p dt = %.3g", c->d.dx,
                          lam_d, wp * c->p.dt);
            delete c;
            return fail(PIC_ERR_UNSTABLE_PARAMS, buf);
        }
    }
    size_t small_end = 0, total = 0;
    carve(c, nullptr, &small_end, &total);
    cudaError_t e = cudaMalloc(&c->arena, total);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaMalloc(state)");
    }
    c->arena_bytes = total;
    c->small_bytes = small_end;
    carve(c, (char*)c->arena, &small_end, &total);
    sync_desc(c);
    cudaDeviceProp prop;
    e = cudaSuccess;
    if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) {
        pic_destroy(c);
        return fail(PIC_ERR_CUDA, "cudaGetDeviceProperties");
    }
    c->sms = prop.multiProcessorCount;
    c->d.trace = nullptr;
    int per_sm = c->p.ctas_per_sm;
    if (per_sm <= 0) {
        e = mover_occupancy(c->d, &per_sm);
        if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    }
    c->grid_mover = c->sms * per_sm;
    if (c->grid_mover > kMaxTallyRows) c->grid_mover = kMaxTallyRows - kMaxTallyRows % c->sms;
    {                                  // the TP step: a multiple of the SMs by its occupancy
        int tp_per_sm = 0, tp_per_sm_sample = 0;
        if (tp_occupancy(c->d, false, &tp_per_sm) != cudaSuccess || tp_per_sm < 1) tp_per_sm = 2;
        if (tp_occupancy(c->d, true, &tp_per_sm_sample) != cudaSuccess || tp_per_sm_sample < 1) tp_per_sm_sample = 2;
        // a launch without the tallies holds at least as many CTAs per SM as one with
        // them (the occupancy query can answer less, for the carveout it assumes)
        c->grid_tp = c->sms * std::max(tp_per_sm, tp_per_sm_sample);
        c->grid_tp_sample = c->sms * tp_per_sm_sample;
    }
    c->grid_sort = c->sms * 8;

    Ctl h;
    std::memset(&h, 0, sizeof h);
    h.n[kE] = c->p.n_e0;
    h.n[kI] = c->p.n_i0;
    h.cap[kE] = c->p.cap_e;
    h.cap[kI] = c->p.cap_i;
    h.cap[kTP] = c->p.cap_tp;
    e = cudaMemsetAsync(c->arena, 0, c->small_bytes, c->stream);
    for (int s = 0; s < 2 && e == cudaSuccess; ++s)
        e = cudaMemsetAsync(c->d.evflag[s], 0, (size_t)(s == kE ? c->p.cap_e : c->p.cap_i) + 4, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d.ctl, &h, sizeof h, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = launch_init(c->d, kE, c->p.n_e0, c->p.id_offset, (float)std::sqrt(c->p.te0_ev * kQE / kME), c->stream);
    if (e == cudaSuccess)
        e = launch_init(c->d, kI, c->p.n_i0, c->p.id_offset, (float)std::sqrt(c->p.ti0_ev * kQE / kMAR), c->stream);
    // the loading is uniform in space but in id order: bring it into cell order
    for (int sp = 0; sp < 2 && e == cudaSuccess; ++sp) {
        if ((sp == kE ? c->p.n_e0 : c->p.n_i0) <= 0) continue;
        e = launch_sort(c->d, sp, c->grid_sort, c->stream);
        c->cur[sp] ^= 1u;
    }
    if (e == cudaSuccess) e = launch_mover(c->d, step_args(c, 0, 0), c->grid_mover, 1, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        pic_destroy(c);
        return cuda_fail(e, "pic_create initial loading");
    }
    *out = c;
    return PIC_OK;
}

void pic_destroy(pic_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto& t : c->timers)
        for (auto ev : t.ev) cudaEventDestroy(ev);
    if (c->arena) cudaFree(c->arena);
    if (c->d.trace) cudaFree(c->d.trace);
    for (float2* t : c->xs_dev)
        if (t) cudaFree(t);
    delete c;
}

int pic_trace(pic_ctx* c, int enable)
{
    if (!c) return fail(PIC_ERR_INVALID_ARG, "ctx is NULL");
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    if (enable && !c->d.trace) {
        unsigned long long* t = nullptr;
        CK(cudaMalloc(&t, (size_t)c->grid_mover * kTraceSlots * 8));
        CK(cudaMemset(t, 0, (size_t)c->grid_mover * kTraceSlots * 8));
        c->d.trace = t;
    } else if (!enable && c->d.trace) {
        CK(cudaFree(c->d.trace));
        c->d.trace = nullptr;
    }
    sync_desc(c);
    return PIC_OK;
}

int pic_trace_read(pic_ctx* c, uint64_t* out, int64_t cap, int64_t* n_written)
{
    if (!c || (!out && cap > 0)) return fail(PIC_ERR_INVALID_ARG, "bad arguments");
    const int64_t n = c->d.trace ? (int64_t)c->grid_mover * kTraceSlots : 0;
    if (n_written) *n_written = n;
    if (n == 0 || cap <= 0) return PIC_OK;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(out, c->d.trace, (size_t)(cap < n ? cap : n) * 8, cudaMemcpyDeviceToHost));
    return PIC_OK;
}

int pic_step(pic_ctx* c, int64_t n)
{
    if (!c || n < 0) return fail(PIC_ERR_INVALID_ARG, "bad context or step count");
    CK(cudaSetDevice(c->device));
    for (int64_t k = 0; k < n; ++k) {
        cudaEvent_t stop;
        int rc = timer_begin(c, 0, &stop);
        if (rc) return rc;
        const int acc = c->h_step > c->acc_upto;
        CK(launch_mover(c->d, step_args(c, c->h_step, acc), c->grid_mover, 0, c->stream));
        if (acc) c->acc_upto = c->h_step;
        rc = timer_end(c, stop);
        if (rc) return rc;
        c->h_step++;
        for (int s = 0; s < 2; ++s) {
            const int every = s == kE ? c->p.sort_every_e : c->p.sort_every_i;
            if (every > 0 && c->h_step % every == 0) {
                rc = timer_begin(c, 2, &stop);
                if (rc) return rc;
                CK(launch_sort(c->d, s, c->grid_sort, c->stream));
                c->cur[s] ^= 1u;
                rc = timer_end(c, stop);
                if (rc) return rc;
            }
        }
        if (c->p.sputter_enable && c->p.tp_every > 0 && c->h_step % c->p.tp_every == 0) {
            rc = run_tp_step(c, c->d_coupled);
            if (rc) return rc;
        }
        if (c->timing && c->timers[0].used >= 4096) {
            CK(cudaStreamSynchronize(c->stream));
            rc = timers_collect(c);
            if (rc) return rc;
        }
    }
    return PIC_OK;
}

int pic_sync(pic_ctx* c)
{
    if (!c) return fail(PIC_ERR_INVALID_ARG, "ctx is NULL");
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    int rc = timers_collect(c);
    if (rc) return rc;
    unsigned int err = 0;
    CK(cudaMemcpy(&err, &c->d.ctl->err, sizeof err, cudaMemcpyDeviceToHost));
    if (err) {
        CK(cudaMemsetAsync(&c->d.ctl->err, 0, sizeof err, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (err & kErrCapacity) return fail(PIC_ERR_CAPACITY, "a birth or launch exceeded the capacity");
        if (err & kErrNumerics) return fail(PIC_ERR_NUMERICS, "electron energy above eps_max");
        if (err & kErrIndex) return fail(PIC_ERR_NUMERICS, "a 64-bit position outside [0, n_cells)");
        if (err & kErrTimeout) return fail(PIC_ERR_TIMEOUT, "a kernel's wait for a bulk copy into shared memory gave up");
    }
    return PIC_OK;
}

int pic_timing(pic_ctx* c, int enable)
{
    if (!c) return fail(PIC_ERR_INVALID_ARG, "ctx is NULL");
    CK(cudaStreamSynchronize(c->stream));
    int rc = timers_collect(c);
    if (rc) return rc;
    for (auto& t : c->timers) {
        t.ms = 0.0;
        t.launches = 0;
    }
    c->timing = enable != 0;
    return PIC_OK;
}

int pic_kernel_time(pic_ctx* c, int kind, double* ms, int64_t* launches)
{
    if (!c || kind < 0 || kind > 2) return fail(PIC_ERR_INVALID_ARG, "bad kind");
    CK(cudaStreamSynchronize(c->stream));
    int rc = timers_collect(c);
    if (rc) return rc;
    if (ms) *ms = c->timers[kind].ms;
    if (launches) *launches = c->timers[kind].launches;
    return PIC_OK;
}

int pic_derived(pic_ctx* c, double* out)
{
    if (!c || !out) return fail(PIC_ERR_INVALID_ARG, "NULL argument");
    std::memcpy(out, c->derived, sizeof c->derived);
    return PIC_OK;
}

static int read_ctl(pic_ctx* c, Ctl* h)
{
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(h, c->d.ctl, sizeof *h, cudaMemcpyDeviceToHost));
    return PIC_OK;
}

// Event counts: the TP kernels' counts in the control block plus the step
// launch's per-CTA rows (d.tally).  tot[kNumCnt].
static int count_events(pic_ctx* c, const Ctl& h, unsigned long long* tot)
{
    std::vector<unsigned long long> rows((size_t)kMaxTallyRows * kNumCnt);
    CK(cudaMemcpy(rows.data(), c->d.tally, rows.size() * 8, cudaMemcpyDeviceToHost));
    for (int k = 0; k < kNumCnt; ++k) tot[k] = h.cnt[k];
    for (size_t r = 0; r < (size_t)kMaxTallyRows; ++r)
        for (int k = 0; k < kNumCnt; ++k) tot[k] += rows[r * kNumCnt + k];
    return PIC_OK;
}

// test particles in flight: launched + sputtered - deposited
static int tp_in_flight(pic_ctx* c, int64_t* n)
{
    Ctl h;
    int rc = read_ctl(c, &h);
    if (rc) return rc;
    unsigned long long tot[kNumCnt];
    if ((rc = count_events(c, h, tot))) return rc;
    *n = c->tp_launched + (int64_t)tot[kCntSputL] + (int64_t)tot[kCntSputR] - (int64_t)tot[kCntTpDepL] -
         (int64_t)tot[kCntTpDepR];
    return PIC_OK;
}

// split sums: word 0 sums the low 32 bits, word 1 the high 32 bits of each added value
static double u128d(const unsigned long long* p) { return (double)p[1] * 4294967296.0 + (double)p[0]; }
static double s128d(const long long* p)
{
    return (double)p[1] * 4294967296.0 + (double)(unsigned long long)p[0];
}

// Potential of a (time-averaged) net charge count qn[0..N] with electrode
// voltage v, by the double prefix sum of the discrete Poisson equation
// (phi[m] = v + m D0 - A sum_{k<m} S_k, S_k = sum_{j=1..k} qn[j]).
static void host_phi(int N, double A, const std::vector<double>& qn, double v, std::vector<double>& phi)
{
    std::vector<long double> S(N + 1), T(N + 1);
    S[0] = 0;
    for (int m = 1; m <= N; ++m) S[m] = S[m - 1] + (long double)qn[m];
    T[0] = 0;
    for (int m = 1; m <= N; ++m) T[m] = T[m - 1] + S[m - 1];
    const long double D0 = (-(long double)v + (long double)A * T[N]) / N;
    phi.resize(N + 1);
    for (int m = 0; m <= N; ++m) phi[m] = (double)((long double)v + m * D0 - (long double)A * T[m]);
}

int pic_diag(pic_ctx* c, int kind, double* out, int64_t cap, int64_t* n_written)
{
    if (!c || (!out && cap > 0) || kind < 0 || kind >= PIC_DIAG_COUNT)
        return fail(PIC_ERR_INVALID_ARG, "bad diag request");
    CK(cudaSetDevice(c->device));
    {                                               // current state into the averages, FP64 field
        const int acc = c->h_step > c->acc_upto;
        CK(launch_field(c->d, field_v_at(c, c->h_step), acc, c->stream));
        if (acc) c->acc_upto = c->h_step;
    }
    Ctl h;
    int rc = read_ctl(c, &h);
    if (rc) return rc;
    const int N = c->p.n_cells, N1 = N + 1;
    const double dx = c->d.dx, w = c->p.weight;
    std::vector<double> v;
    auto getd = [&](const double* src, size_t n, std::vector<double>& dst) -> int {
        dst.resize(n);
        CK(cudaMemcpy(dst.data(), src, n * sizeof(double), cudaMemcpyDeviceToHost));
        return PIC_OK;
    };
    auto getu = [&](const unsigned long long* src, size_t n, std::vector<double>& dst) -> int {
        std::vector<unsigned long long> t(n);
        CK(cudaMemcpy(t.data(), src, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
        dst.assign(t.begin(), t.end());
        return PIC_OK;
    };
    auto getu128 = [&](const unsigned long long* src, std::vector<double>& dst) -> int {
        std::vector<unsigned long long> t(2 * (size_t)N1);
        CK(cudaMemcpy(t.data(), src, t.size() * 8, cudaMemcpyDeviceToHost));
        dst.resize(N1);
        for (int m = 0; m < N1; ++m) dst[m] = u128d(&t[2 * m]);
        return PIC_OK;
    };
    auto gets128 = [&](const long long* src, std::vector<double>& dst) -> int {
        std::vector<long long> t(2 * (size_t)N1);
        CK(cudaMemcpy(t.data(), src, t.size() * 8, cudaMemcpyDeviceToHost));
        dst.resize(N1);
        for (int m = 0; m < N1; ++m) dst[m] = s128d(&t[2 * m]);
        return PIC_OK;
    };
    auto vol = [&](int m) { return (m == 0 || m == N) ? 0.5 * dx : dx; };
    const double navg = h.n_avg ? (double)h.n_avg : 1.0, nflux = h.n_flux ? (double)h.n_flux : 1.0;
    std::vector<double> a, b;
    switch (kind) {
    case PIC_DIAG_PHI: {
        if ((rc = getu128(c->d.diag.sum_q[kE], a))) return rc;
        if ((rc = getu128(c->d.diag.sum_q[kI], b))) return rc;
        std::vector<double> qn(N1);
        for (int m = 0; m < N1; ++m) qn[m] = (b[m] - a[m]) / navg;
        host_phi(N, c->d.A, qn, h.sum_v / navg, v);
        if (!h.n_avg) std::fill(v.begin(), v.end(), 0.0);
        break;
    }
    case PIC_DIAG_NE: case PIC_DIAG_NI:
        if ((rc = getu128(c->d.diag.sum_q[kind - PIC_DIAG_NE], v))) return rc;
        for (int m = 0; m < N1; ++m) v[m] = h.n_avg ? w * v[m] / (4294967296.0 * vol(m) * navg) : 0.0;
        break;
    case PIC_DIAG_GAMMA_E: case PIC_DIAG_GAMMA_I:
        if ((rc = gets128(c->d.diag.sum_flux[kind - PIC_DIAG_GAMMA_E], v))) return rc;
        for (int m = 0; m < N1; ++m) v[m] = h.n_flux ? w * v[m] * 0x1p-16 / (vol(m) * nflux) : 0.0;
        break;
    case PIC_DIAG_VE: case PIC_DIAG_VI: {
        const int s = kind - PIC_DIAG_VE;
        if ((rc = gets128(c->d.diag.sum_flux[s], a))) return rc;
        if ((rc = getu128(c->d.diag.sum_q[s], b))) return rc;
        v.resize(N1);
        for (int m = 0; m < N1; ++m) {
            // Gamma / n with both averages: (sum_flux 2^-16 / n_flux) / (sum_q 2^-32 / n_avg)
            const double nq = b[m] * 0x1p-32 / navg;
            v[m] = (h.n_flux && nq > 0) ? (a[m] * 0x1p-16 / nflux) / nq : 0.0;
        }
        break;
    }
    case PIC_DIAG_EEDF:
        if ((rc = getu(c->d.diag.eedf, kNbEedf, v))) return rc;
        break;
    case PIC_DIAG_IEDF_L: case PIC_DIAG_IEDF_R:
        if ((rc = getu(c->d.diag.iedf[kind - PIC_DIAG_IEDF_L], kNbIedf, v))) return rc;
        break;
    case PIC_DIAG_IEADF_L: case PIC_DIAG_IEADF_R:
        if ((rc = getu(c->d.diag.ieadf[kind - PIC_DIAG_IEADF_L], kNbIeadfE * kNbAng, v))) return rc;
        break;
    case PIC_DIAG_SPUTTER_E_L: case PIC_DIAG_SPUTTER_E_R:
        if ((rc = getu(c->d.diag.sp_e[kind - PIC_DIAG_SPUTTER_E_L], kNbSpE, v))) return rc;
        break;
    case PIC_DIAG_SPUTTER_ANG_L: case PIC_DIAG_SPUTTER_ANG_R:
        if ((rc = getu(c->d.diag.sp_ang[kind - PIC_DIAG_SPUTTER_ANG_L], kNbAng, v))) return rc;
        break;
    case PIC_DIAG_TP_DENS:
        if ((rc = getu128(c->d.diag.tp_dens, v))) return rc;
        for (int m = 0; m < N1; ++m)
            v[m] = h.n_tp_samp ? w * v[m] * 0x1p-32 / (vol(m) * (double)h.n_tp_samp) : 0.0;
        break;
    case PIC_DIAG_TP_V:
        if ((rc = gets128(c->d.diag.tp_vx, a))) return rc;
        if ((rc = getu128(c->d.diag.tp_dens, b))) return rc;
        v.resize(N1);
        for (int m = 0; m < N1; ++m) v[m] = b[m] > 0 ? (a[m] * 0x1p-16) / (b[m] * 0x1p-32) : 0.0;
        break;
    case PIC_DIAG_E:
        if ((rc = getd(c->d.E64, N1, v))) return rc;
        break;
    case PIC_DIAG_PHI_NOW:
        if ((rc = getd(c->d.phi, N1, v))) return rc;
        break;
    case PIC_DIAG_TPF_TIME: case PIC_DIAG_TPF_VX: {
        std::vector<long long> tp(N1), td(N1), dp(N1), dd(N1);
        CK(cudaMemcpy(tp.data(), c->d.diag.tpf_tpart, N1 * 8, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(td.data(), c->d.diag.tpf_tdiff, N1 * 8, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(dp.data(), c->d.diag.tpf_dpart, N1 * 8, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(dd.data(), c->d.diag.tpf_ddiff, N1 * 8, cudaMemcpyDeviceToHost));
        v.assign(N, 0.0);
        long long ts = 0, ds = 0;
        for (int j = 0; j < N; ++j) {
            ts += td[j];
            ds += dd[j];
            const double t = (double)(tp[j] + ts) * 0x1p-40;             // s
            const double path = (double)(dp[j] + ds) * (c->p.gap_m * 0x1p-32);   // m
            v[j] = kind == PIC_DIAG_TPF_TIME ? t : (t > 0.0 ? path / t : 0.0);
        }
        break;
    }
    }
    const int64_t n = (int64_t)v.size();
    for (int64_t i = 0; i < n && i < cap; ++i) out[i] = v[i];
    if (n_written) *n_written = n;
    return PIC_OK;
}

int pic_hypotheses(pic_ctx* c, double* out)
{
    if (!c || !out) return fail(PIC_ERR_INVALID_ARG, "NULL argument");
    const int N1 = c->p.n_cells + 1;
    std::vector<double> h(kNbIeadfE * kNbAng > N1 ? kNbIeadfE * kNbAng : N1);
    int64_t n = 0;
    for (int el = 0; el < 2; ++el) {
        // width-to-peak of the ion energy distribution: the fullest bin (the
        // first of equals) and the run of bins around it at or above half of it
        int rc = pic_diag(c, PIC_DIAG_IEDF_L + el, h.data(), (int64_t)h.size(), &n);
        if (rc) return rc;
        int pk = 0;
        for (int b = 1; b < kNbIedf; ++b)
            if (h[b] > h[pk]) pk = b;
        double r = 0.0;
        if (h[pk] > 0.0) {
            int lo = pk, hi = pk;
            while (lo > 0 && h[lo - 1] >= 0.5 * h[pk]) --lo;
            while (hi < kNbIedf - 1 && h[hi + 1] >= 0.5 * h[pk]) ++hi;
            r = (double)(hi - lo + 1) / (pk + 0.5);
        }
        out[el] = r;
        // rms impact angle over the energy-summed angle histogram (bin centres)
        rc = pic_diag(c, PIC_DIAG_IEADF_L + el, h.data(), (int64_t)h.size(), &n);
        if (rc) return rc;
        double s0 = 0.0, s2 = 0.0;
        for (int b = 0; b < kNbAng; ++b) {
            double col = 0.0;
            for (int e = 0; e < kNbIeadfE; ++e) col += h[(size_t)e * kNbAng + b];
            s0 += col;
            s2 += col * (b + 0.5) * (b + 0.5);
        }
        out[2 + el] = s0 > 0.0 ? std::sqrt(s2 / s0) : 0.0;
    }
    const double ngas = c->derived[0];
    for (int k = 0; k < 2; ++k) {
        int rc = pic_diag(c, k == 0 ? PIC_DIAG_NI : PIC_DIAG_TP_DENS, h.data(), (int64_t)h.size(), &n);
        if (rc) return rc;
        double mx = 0.0;
        for (int m = 0; m < N1; ++m) mx = std::max(mx, h[m]);
        out[4 + k] = ngas > 0.0 ? mx / ngas : 0.0;
    }
    return PIC_OK;
}

int pic_reset_averages(pic_ctx* c)
{
    if (!c) return fail(PIC_ERR_INVALID_ARG, "ctx is NULL");
    CK(cudaSetDevice(c->device));
    const int N1 = c->p.n_cells + 1;
    const Diag& g = c->d.diag;
    for (int s = 0; s < 2; ++s) {
        CK(cudaMemsetAsync(g.sum_q[s], 0, 2 * N1 * 8, c->stream));
        CK(cudaMemsetAsync(g.sum_flux[s], 0, 2 * N1 * 8, c->stream));
        CK(cudaMemsetAsync(g.iedf[s], 0, kNbIedf * 8, c->stream));
        CK(cudaMemsetAsync(g.ieadf[s], 0, kNbIeadfE * kNbAng * 8, c->stream));
        CK(cudaMemsetAsync(g.sp_e[s], 0, kNbSpE * 8, c->stream));
        CK(cudaMemsetAsync(g.sp_ang[s], 0, kNbAng * 8, c->stream));
    }
    CK(cudaMemsetAsync(g.tp_dens, 0, 2 * N1 * 8, c->stream));
    for (long long* a : {g.tpf_tpart, g.tpf_tdiff, g.tpf_dpart, g.tpf_ddiff})
        CK(cudaMemsetAsync(a, 0, N1 * 8, c->stream));
    CK(cudaMemsetAsync(g.tp_vx, 0, 2 * N1 * 8, c->stream));
    CK(cudaMemsetAsync(g.eedf, 0, kNbEedf * 8, c->stream));
    CK(cudaMemsetAsync(&c->d.ctl->n_avg, 0, 3 * sizeof(long long), c->stream));
    CK(cudaMemsetAsync(&c->d.ctl->sum_v, 0, sizeof(double), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->acc_upto = c->h_step;           // the current state is not part of the new window
    return PIC_OK;
}

int pic_counters(pic_ctx* c, int64_t* out, int64_t cap, int64_t* n_written)
{
    if (!c || (!out && cap > 0)) return fail(PIC_ERR_INVALID_ARG, "bad arguments");
    CK(cudaSetDevice(c->device));
    Ctl h;
    int rc = read_ctl(c, &h);
    if (rc) return rc;
    int64_t v[5 + kNumCnt];
    v[0] = h.n[kE]; v[1] = h.n[kI]; v[2] = h.n[kTP]; v[3] = h.step; v[4] = h.tp_step;
    // order: impacts e L/R, Ar+ L/R, ionisations, sputtered L/R, Al deposited L/R,
    // numerics, elastic, excitation, CX, isotropic, TP collisions, capacity
    const int order[kNumCnt] = {kCntImpEL, kCntImpER, kCntImpIL, kCntImpIR, kCntIoniz, kCntSputL,
                                kCntSputR, kCntTpDepL, kCntTpDepR, kCntNumerics, kCntElastic,
                                kCntExcit, kCntCx, kCntIso, kCntTpColl, kCntCapacity};
    // the step launch keeps its counts per CTA (rows of d.tally)
    unsigned long long tot[kNumCnt];
    if ((rc = count_events(c, h, tot))) return rc;
    for (int i = 0; i < kNumCnt; ++i) v[5 + i] = (int64_t)tot[order[i]];
    const int64_t n = 5 + kNumCnt;
    for (int64_t i = 0; i < n && i < cap; ++i) out[i] = v[i];
    if (n_written) *n_written = n;
    return PIC_OK;
}

int pic_get_species(pic_ctx* c, int s, int64_t cap, double* xi, float* vx, float* vy, float* vz,
                    uint64_t* id, int64_t* n_out)
{
    if (!c || s < 0 || s > 2 || cap < 0) return fail(PIC_ERR_INVALID_ARG, "bad arguments");
    CK(cudaSetDevice(c->device));
    Ctl h;
    int rc = read_ctl(c, &h);
    if (rc) return rc;
    const long long n = h.n[s];
    const SpBuf& B = c->d.buf[s][h.cur[s]];
    const bool p64 = c->p.pos_precision == 64 && s != kTP;
    std::vector<unsigned char> pos((size_t)n * (p64 ? 8 : 4));
    std::vector<float> a((size_t)n), b((size_t)n), cc((size_t)n);
    std::vector<uint64_t> ids((size_t)n);
    if (n > 0) {
        CK(cudaMemcpy(pos.data(), B.pos, pos.size(), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(a.data(), B.vx, n * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(b.data(), B.vy, n * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(cc.data(), B.vz, n * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(ids.data(), B.id, n * 8, cudaMemcpyDeviceToHost));
    }
    const double scale = (double)c->p.n_cells * 0x1p-32;
    int64_t m = 0;
    for (long long k = 0; k < n; ++k) {
        double x;
        if (p64) {
            x = ((const double*)pos.data())[k];
            if (!(x >= 0.0)) continue;
        } else {
            const uint32_t u = ((const uint32_t*)pos.data())[k];
            if (u == 0) continue;
            x = (double)u * scale;
        }
        if (m < cap) {
            if (xi) xi[m] = x;
            if (vx) vx[m] = a[k];
            if (vy) vy[m] = b[k];
            if (vz) vz[m] = cc[k];
            if (id) id[m] = ids[k];
        }
        ++m;
    }
    if (n_out) *n_out = m;
    return PIC_OK;
}

int pic_set_species(pic_ctx* c, int s, int64_t n, const void* pos, const float* vx, const float* vy,
                    const float* vz, const uint64_t* id, int keep_field)
{
    if (!c || s < 0 || s > 2 || n < 0 || (n > 0 && (!pos || !vx || !vy || !vz || !id)))
        return fail(PIC_ERR_INVALID_ARG, "bad arguments");
    const long long cap = s == kE ? c->p.cap_e : (s == kI ? c->p.cap_i : c->p.cap_tp);
    if (n > cap) return fail(PIC_ERR_CAPACITY, "more particles than the species capacity");
    CK(cudaSetDevice(c->device));
    Ctl h;
    int rc = read_ctl(c, &h);
    if (rc) return rc;
    const SpBuf& B = c->d.buf[s][h.cur[s]];
    const bool p64 = c->p.pos_precision == 64 && s != kTP;
    if (n > 0) {
        CK(cudaMemcpyAsync(B.pos, pos, (size_t)n * (p64 ? 8 : 4), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(B.vx, vx, (size_t)n * 4, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(B.vy, vy, (size_t)n * 4, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(B.vz, vz, (size_t)n * 4, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(B.id, id, (size_t)n * 8, cudaMemcpyHostToDevice, c->stream));
        if (s != kTP) CK(launch_entry_nev(c->d, s, h.cur[s], n, (unsigned int)c->h_step, c->stream));
        else CK(cudaMemsetAsync(B.nev, 0, (size_t)n * 4, c->stream));   // no flight event yet
    }
    long long nn = n;
    CK(cudaMemcpyAsync(&c->d.ctl->n[s], &nn, sizeof nn, cudaMemcpyHostToDevice, c->stream));
    if (!keep_field && s != kTP) {      // re-deposit the state of the current step
        const int slot = h.step % 3;
        const size_t N1 = (size_t)c->p.n_cells + 1;
        CK(cudaMemsetAsync(c->d.qbuf[slot][kE], 0, N1 * 8, c->stream));
        CK(cudaMemsetAsync(c->d.qbuf[slot][kI], 0, N1 * 8, c->stream));
        CK(launch_mover(c->d, step_args(c, c->h_step, 0), c->grid_mover, 1, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

int pic_get_field(pic_ctx* c, double* E, double* phi, int64_t* q_e, int64_t* q_i)
{
    if (!c) return fail(PIC_ERR_INVALID_ARG, "ctx is NULL");
    CK(cudaSetDevice(c->device));
    CK(launch_field(c->d, field_v_at(c, c->h_step), 0, c->stream));
    Ctl h;
    int rc = read_ctl(c, &h);
    if (rc) return rc;
    const size_t N1 = (size_t)c->p.n_cells + 1;
    const int slot = h.step % 3;
    if (E) CK(cudaMemcpy(E, c->d.E64, N1 * 8, cudaMemcpyDeviceToHost));
    if (phi) CK(cudaMemcpy(phi, c->d.phi, N1 * 8, cudaMemcpyDeviceToHost));
    if (q_e) CK(cudaMemcpy(q_e, c->d.qbuf[slot][kE], N1 * 8, cudaMemcpyDeviceToHost));
    if (q_i) CK(cudaMemcpy(q_i, c->d.qbuf[slot][kI], N1 * 8, cudaMemcpyDeviceToHost));
    return PIC_OK;
}

int pic_set_field(pic_ctx* c, const double* E)
{
    if (!c || !E) return fail(PIC_ERR_INVALID_ARG, "NULL argument");
    CK(cudaSetDevice(c->device));
    const size_t N1 = (size_t)c->p.n_cells + 1;
    std::vector<float> f(N1);
    for (size_t m = 0; m < N1; ++m) f[m] = (float)E[m];
    const unsigned int one = 1;
    CK(cudaMemcpyAsync(c->d.E32, f.data(), N1 * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(&c->d.ctl->field_override, &one, sizeof one, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

int tp_launch(pic_ctx* c, const tp_source* src)
{
    if (!c || !src || src->n < 0 || !(src->e_ion_ev >= 0)) return fail(PIC_ERR_INVALID_ARG, "bad source");
    if (src->first_id >= 0 && src->first_id + src->n > (1ll << 61))
        return fail(PIC_ERR_INVALID_ARG, "source ids must stay below 2^61");
    CK(cudaSetDevice(c->device));
    const float Emax = (float)(c->derived[7] * src->e_ion_ev);
    CK(launch_tp_launch(c->d, src->n, src->first_id >= 0 ? src->first_id : c->tp_launched, Emax, c->stream));
    c->tp_launched += src->n;
    return PIC_OK;
}

int pic_test_wait_timeout(pic_ctx* c, int enable)
{
    if (!c) return fail(PIC_ERR_INVALID_ARG, "ctx is NULL");
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    c->d.tp_wait_test = enable ? 1 : 0;
    c->d.tp_wait_spin = enable ? 4096u : (1u << 22);
    sync_desc(c);
    return PIC_OK;
}

int pic_exchange_slot(pic_ctx* c, int64_t** dev, int64_t* n_words)
{
    if (!c || !dev || !n_words) return fail(PIC_ERR_INVALID_ARG, "NULL argument");
    if (c->p.circuit) return fail(PIC_ERR_INVALID_ARG, "the series capacitor needs the whole wall charge: "
                                                       "no split discharge with circuit 1");
    const int slot = (int)(c->h_step % 3);
    *dev = (int64_t*)c->d.qbuf[slot][0];
    *n_words = 4 * c->exch_stride;
    return PIC_OK;
}

int tp_step(pic_ctx* c, int64_t n, int64_t* n_alive)
{
    if (!c || n < 0) return fail(PIC_ERR_INVALID_ARG, "bad arguments");
    CK(cudaSetDevice(c->device));
    for (int64_t k = 0; k < n; ++k) {
        int rc = run_tp_step(c, c->d);
        if (rc) return rc;
    }
    if (n_alive) {
        int rc = tp_in_flight(c, n_alive);
        if (rc) return rc;
    }
    return PIC_OK;
}

int tp_flight(pic_ctx* c, int64_t max_events, int64_t* n_alive)
{
    if (!c || max_events < 0) return fail(PIC_ERR_INVALID_ARG, "bad arguments");
    CK(cudaSetDevice(c->device));
    constexpr int kEventsPerLaunch = 32;
    unsigned long long alive = 0;
    bool any = false;
    for (int64_t done = 0; done < max_events;) {
        const int k = (int)std::min<int64_t>(kEventsPerLaunch, max_events - done);
        CK(cudaMemsetAsync(&c->d.ctl->tpf_alive, 0, sizeof(unsigned long long), c->stream));
        Ctl h;                                         // slots in use: the launch takes one CTA per 1024
        CK(cudaMemcpy(&h.n[kTP], &c->d.ctl->n[kTP], sizeof(long long), cudaMemcpyDeviceToHost));
        CK(launch_tp_flight(c->d, k, h.n[kTP], c->stream));
        CK(cudaMemcpyAsync(&alive, &c->d.ctl->tpf_alive, sizeof alive, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        any = true;
        done += k;
        if (alive == 0) break;
    }
    if (n_alive) {
        if (!any) {                                    // no launch: count the live atoms as they are
            int64_t n = 0;
            int rc = tp_in_flight(c, &n);
            if (rc) return rc;
            alive = (unsigned long long)n;
        }
        *n_alive = (int64_t)alive;
    }
    return PIC_OK;
}

int pic_set_cross_section(pic_ctx* c, int q, int64_t n, const double* E, const double* sigma)
{
    if (!c || q < 0 || q > 2 || n < 0 || n == 1 || n > 65536 || (n > 0 && (!E || !sigma)))
        return fail(PIC_ERR_INVALID_ARG, "process 0..2 and a table of 0 or 2..65536 points");
    for (int64_t i = 0; i < n; ++i)
        if (!(sigma[i] >= 0.0) || !std::isfinite(E[i]) || (i > 0 && !(E[i] > E[i - 1])))
            return fail(PIC_ERR_INVALID_ARG, "energies must increase and cross sections be >= 0");
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    if (c->xs_dev[q]) CK(cudaFree(c->xs_dev[q]));
    c->xs_dev[q] = nullptr;
    c->xs_e[q].assign(E, E + n);
    c->xs_s[q].assign(sigma, sigma + n);
    if (n) {
        std::vector<float2> t((size_t)n);
        for (int64_t i = 0; i < n; ++i) t[(size_t)i] = make_float2((float)E[i], (float)sigma[i]);
        CK(cudaMalloc(&c->xs_dev[q], sizeof(float2) * (size_t)n));
        CK(cudaMemcpy(c->xs_dev[q], t.data(), sizeof(float2) * (size_t)n, cudaMemcpyHostToDevice));
    }
    c->d.xs_tab[q] = c->xs_dev[q];
    c->d.xs_n[q] = (int)n;
    derive(c);                                      // nu_max of the electrons from the tables
    // the candidate process is memoryless: every electron's next candidate is
    // drawn afresh from the current step at the new nu_max
    Ctl h;
    int rc = read_ctl(c, &h);
    if (rc) return rc;
    CK(launch_entry_nev(c->d, kE, h.cur[kE], h.n[kE], (unsigned int)c->h_step, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

int pic_compact(pic_ctx* c, int s)
{
    if (!c || s < 0 || s > 2) return fail(PIC_ERR_INVALID_ARG, "bad species");
    CK(cudaSetDevice(c->device));
    CK(launch_sort(c->d, s, c->grid_sort, c->stream));
    c->cur[s] ^= 1u;
    return PIC_OK;
}

int pic_op_deposit(const void* pos, int prec, int64_t n, int32_t n_cells, int64_t* q, void* stream)
{
    if ((!pos && n > 0) || !q || n < 0 || (prec != 32 && prec != 64) || !pow2(n_cells) || n_cells < 4 ||
        n_cells > 4096)
        return fail(PIC_ERR_INVALID_ARG, "bad deposit arguments");
    if (n == 0) return PIC_OK;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    long long g = (n + 2047) / 2048;
    if (g > sms * 4) g = sms * 4;
    CK(launch_op_deposit(pos, prec == 64, n, n_cells, ilog2(n_cells), (unsigned long long*)q, (int)g,
                         (cudaStream_t)stream));
    return PIC_OK;
}

int pic_op_poisson(const int64_t* q_i, const int64_t* q_e, int32_t n_cells, double dx, double w,
                   double v_left, double* phi, double* E, void* stream)
{
    if (!q_i || !q_e || n_cells < 2 || n_cells > 1 << 20 || !(dx > 0)) return fail(PIC_ERR_INVALID_ARG, "bad poisson arguments");
    const double A = dx * kQE * w / (4294967296.0 * kEPS0);
    CK(launch_op_poisson((const long long*)q_i, (const long long*)q_e, n_cells, A, 1.0 / dx, v_left, phi,
                         E, (cudaStream_t)stream));
    return PIC_OK;
}

const char* pic_strerror(int code)
{
    switch (code) {
    case PIC_OK: return "ok";
    case PIC_ERR_INVALID_ARG: return "invalid argument";
    case PIC_ERR_UNSTABLE_PARAMS: return "parameters violate dx < lambda_D or w_p dt < 1";
    case PIC_ERR_OUT_OF_MEMORY: return "device out of memory";
    case PIC_ERR_CAPACITY: return "particle capacity exceeded";
    case PIC_ERR_NUMERICS: return "electron energy above the null-collision bound";
    case PIC_ERR_CUDA: return "CUDA error";
    case PIC_ERR_NO_DEVICE: return "no CUDA device";
    case PIC_ERR_TIMEOUT: return "timed out";
    default: return "unknown error";
    }
}

const char* pic_last_error(void) { return g_err.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------- batches
struct pic_batch {
    std::vector<pic_ctx*> ctx;             // slots; nullptr where a discharge was removed
    std::vector<StepArgs*> phase;          // per slot: device table of the step arguments of one RF period
    cudaStream_t stream = nullptr;
    long long target = 0;                  // particles per CTA of the batched launch; 0: automatic
    BatchEntry* d_ent = nullptr;
    int* d_owner = nullptr;
    size_t ent_cap = 0, owner_cap = 0;
    std::vector<BatchEntry> h_ent;
    std::vector<int> h_owner;
    int grid = 0, max_ncell = 0;
    bool dirty = true;
    // resident-CTA launch: chunks of CTA slots taken from a work counter
    long long chunk = 131072;              // particles per chunk; 0: one CTA per slot
    std::vector<BatchChunk> h_chunk;
    BatchChunk* d_chunk = nullptr;
    size_t chunk_cap = 0;
    unsigned int* d_work = nullptr;
    int grid_res = 0;                      // resident CTAs of the chunked launch
    // CUDA graph of one sampling period (diag_every launches), replayed while
    // no compaction falls inside it; captured on a private stream
    bool use_graph = false;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    // optional event pairs around each launch or graph replay, with the steps each covers
    bool timing = false;
    std::vector<cudaEvent_t> tev;
    std::vector<int> tsteps;
    size_t tused = 0;
    double t_ms = 0.0;
    long long t_steps = 0;
};

namespace {

int batch_rebuild(pic_batch* b)
{
    b->h_ent.clear();
    b->h_owner.clear();
    b->max_ncell = 0;
    long long total = 0;
    for (pic_ctx* c : b->ctx)
        if (c) {
            b->max_ncell = std::max(b->max_ncell, c->p.n_cells);
            total += c->p.n_e0 + c->p.n_i0;
        }
    int per_sm = 0;
    if (b->max_ncell > 0) CK(mover_batch_attr(b->max_ncell, &per_sm));
    long long target = b->target;
    if (target <= 0) {
        // automatic: at least two waves of resident CTAs, at most 16384
        // particles per CTA (the best division the autotuner found for a
        // launch of many waves), at least 2048
        int dev = 0, sms = 1;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const long long slots = (long long)sms * std::max(per_sm, 1);
        target = std::min(16384ll, std::max(2048ll, (total + 2 * slots - 1) / (2 * slots)));
    }
    int cta = 0;
    for (size_t k = 0; k < b->ctx.size(); ++k) {
        pic_ctx* c = b->ctx[k];
        if (!c) continue;
        const long long np = c->p.n_e0 + c->p.n_i0;
        const int ncta = (int)std::max(2ll, (np + target - 1) / target);
        BatchEntry e;
        std::memset(&e, 0, sizeof e);
        e.d = c->d;
        e.phase = b->phase[k];
        e.period = (unsigned int)c->period;
        e.cta0 = cta;
        e.ncta = ncta;
        b->h_ent.push_back(e);
        for (int i = 0; i < ncta; ++i) b->h_owner.push_back((int)b->h_ent.size() - 1);
        cta += ncta;
    }
    b->grid = cta;
    // chunks of consecutive CTA slots of one member; the last fifth of each
    // member's slots go, one per chunk, to the end of the list, so the launch
    // ends on short pieces of work.  A chunk holds at most a 2R-th of all
    // slots (R resident CTAs), so that a small batch -- a request loop holds
    // a few discharges -- still spreads over the whole GPU
    int dev = 0, sms = 1;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long resident = (long long)sms * std::max(per_sm, 1);
    const long long per_cap = std::max(1ll, (long long)b->grid / (2 * resident));
    b->h_chunk.clear();
    std::vector<BatchChunk> tail;
    for (size_t k = 0; k < b->h_ent.size(); ++k) {
        const int ncta = b->h_ent[k].ncta;
        const int per = (int)std::max(1ll, std::min(b->chunk / std::max(1ll, target), per_cap));
        const int head = per > 1 ? (ncta * 4 / 5) / per * per : ncta;
        for (int v = 0; v < head; v += per) b->h_chunk.push_back(BatchChunk{(int)k, v, std::min(head, v + per), 0});
        for (int v = head; v < ncta; ++v) tail.push_back(BatchChunk{(int)k, v, v + 1, 0});
    }
    b->h_chunk.insert(b->h_chunk.end(), tail.begin(), tail.end());
    b->grid_res = (int)std::min<long long>(resident, (long long)b->h_chunk.size());
    if (b->h_chunk.size() > b->chunk_cap) {
        if (b->d_chunk) CK(cudaFree(b->d_chunk));
        b->d_chunk = nullptr;
        b->chunk_cap = b->h_chunk.size() + 256;
        CK(cudaMalloc(&b->d_chunk, b->chunk_cap * sizeof(BatchChunk)));
    }
    if (!b->d_work) {
        CK(cudaMalloc(&b->d_work, 2 * sizeof(unsigned int)));
        CK(cudaMemsetAsync(b->d_work, 0, 2 * sizeof(unsigned int), b->stream));
    }
    if (!b->h_chunk.empty())
        CK(cudaMemcpyAsync(b->d_chunk, b->h_chunk.data(), b->h_chunk.size() * sizeof(BatchChunk),
                           cudaMemcpyHostToDevice, b->stream));
    if (b->gexec) {
        CK(cudaGraphExecDestroy(b->gexec));
        b->gexec = nullptr;
    }
    if (b->h_ent.size() > b->ent_cap) {
        if (b->d_ent) CK(cudaFree(b->d_ent));
        b->d_ent = nullptr;
        b->ent_cap = b->h_ent.size() + 16;
        CK(cudaMalloc(&b->d_ent, b->ent_cap * sizeof(BatchEntry)));
    }
    if (b->h_owner.size() > b->owner_cap) {
        if (b->d_owner) CK(cudaFree(b->d_owner));
        b->d_owner = nullptr;
        b->owner_cap = b->h_owner.size() + 256;
        CK(cudaMalloc(&b->d_owner, b->owner_cap * sizeof(int)));
    }
    if (!b->h_owner.empty())
        CK(cudaMemcpyAsync(b->d_owner, b->h_owner.data(), b->h_owner.size() * sizeof(int), cudaMemcpyHostToDevice,
                           b->stream));
    b->dirty = false;
    return PIC_OK;
}

// After one step of the batch: host step counts and each member's due compactions.
int batch_advance(pic_batch* b)
{
    for (pic_ctx* c : b->ctx) {
        if (!c) continue;
        c->acc_upto = c->h_step;
        c->h_step++;
        for (int s = 0; s < 2; ++s) {
            const int every = s == kE ? c->p.sort_every_e : c->p.sort_every_i;
            if (every > 0 && c->h_step % every == 0) {
                CK(launch_sort(c->d, s, c->grid_sort, b->stream));
                c->cur[s] ^= 1u;
            }
        }
    }
    return PIC_OK;
}

// one step launch of every member: resident CTAs taking chunks, or one CTA per slot
cudaError_t batch_launch(pic_batch* b, bool sample, cudaStream_t st)
{
    if (b->chunk > 0)
        return launch_mover_batch_chunks(b->d_ent, b->d_chunk, (int)b->h_chunk.size(), b->d_work, b->grid_res,
                                         b->max_ncell, sample, st);
    return launch_mover_batch(b->d_ent, b->d_owner, b->grid, b->max_ncell, sample, st);
}

// Whether a member compacts after one of the first m - 1 steps from step l on.
bool batch_sort_inside(const pic_batch* b, long long l, int m)
{
    for (const pic_ctx* c : b->ctx) {
        if (!c) continue;
        for (int s = 0; s < 2; ++s) {
            const int every = s == kE ? c->p.sort_every_e : c->p.sort_every_i;
            if (every <= 0) continue;
            for (int j = 1; j < m; ++j)
                if ((l + j) % every == 0) return true;
        }
    }
    return false;
}

// Capture m step launches (the last one sampling) into the batch's graph.
int batch_capture(pic_batch* b, int m)
{
    if (!b->cap_stream) CK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < m && e == cudaSuccess; ++j) e = batch_launch(b, j == m - 1, b->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->gexec = nullptr;
        return cuda_fail(e, "batch graph capture");
    }
    return PIC_OK;
}

int batch_timers_collect(pic_batch* b)
{
    for (size_t i = 0; i + 1 < b->tused; i += 2) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, b->tev[i], b->tev[i + 1]));
        b->t_ms += ms;
        b->t_steps += b->tsteps[i / 2];
    }
    b->tused = 0;
    return PIC_OK;
}

// begin: record the start of a timed launch covering `steps` steps; else its end.
int batch_timer(pic_batch* b, int steps, bool begin)
{
    if (!b->timing) return PIC_OK;
    if (begin) {
        if (b->tused + 2 > b->tev.size()) {
            for (int i = 0; i < 64; ++i) {
                cudaEvent_t ev;
                CK(cudaEventCreate(&ev));
                b->tev.push_back(ev);
            }
        }
        b->tsteps.resize(b->tev.size() / 2);
        b->tsteps[b->tused / 2] = steps;
    }
    CK(cudaEventRecord(b->tev[b->tused], b->stream));
    ++b->tused;
    if (!begin && b->tused >= 4096) {
        CK(cudaStreamSynchronize(b->stream));
        return batch_timers_collect(b);
    }
    return PIC_OK;
}

}  // namespace

extern "C" {

int pic_batch_create(void* stream, pic_batch** out)
{
    if (!out) return fail(PIC_ERR_INVALID_ARG, "out is NULL");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(PIC_ERR_NO_DEVICE, "no CUDA device");
    pic_batch* b = new pic_batch();
    b->stream = (cudaStream_t)stream;
    *out = b;
    return PIC_OK;
}

int pic_batch_add(pic_batch* b, const pic_params* p, int* slot)
{
    if (!b || !p || !slot) return fail(PIC_ERR_INVALID_ARG, "bad arguments");
    if (p->pos_precision != 32) return fail(PIC_ERR_INVALID_ARG, "batched discharges use 32-bit positions");
    if (p->sputter_enable && p->tp_every > 0)
        return fail(PIC_ERR_INVALID_ARG, "batched discharges run no coupled test-particle steps (tp_every 0)");
    for (pic_ctx* o : b->ctx) {
        if (!o) continue;
        if (o->p.dt != p->dt || o->p.diag_every != p->diag_every)
            return fail(PIC_ERR_INVALID_ARG, "a batch shares one dt and one diag_every");
        if (o->p.diag_every > 0 && o->h_step % o->p.diag_every != 0)
            return fail(PIC_ERR_INVALID_ARG, "discharges join a batch at a multiple of diag_every steps");
        break;
    }
    pic_ctx* c = nullptr;
    int rc = pic_create(p, b->stream, &c);
    if (rc) return rc;
    if (c->period <= 0) {
        pic_destroy(c);
        return fail(PIC_ERR_INVALID_ARG, "batched discharges need a whole number of steps per RF period");
    }
    std::vector<StepArgs> tab((size_t)c->period);
    for (long long l = 0; l < c->period; ++l) tab[(size_t)l] = step_args(c, l, 1);
    StepArgs* dt = nullptr;
    cudaError_t e = cudaMalloc(&dt, tab.size() * sizeof(StepArgs));
    if (e == cudaSuccess)
        e = cudaMemcpy(dt, tab.data(), tab.size() * sizeof(StepArgs), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (dt) cudaFree(dt);
        pic_destroy(c);
        return cuda_fail(e, "batch phase table");
    }
    size_t k = 0;
    while (k < b->ctx.size() && b->ctx[k]) ++k;
    if (k == b->ctx.size()) {
        b->ctx.push_back(nullptr);
        b->phase.push_back(nullptr);
    }
    b->ctx[k] = c;
    b->phase[k] = dt;
    b->dirty = true;
    *slot = (int)k;
    return PIC_OK;
}

int pic_batch_remove(pic_batch* b, int slot)
{
    if (!b || slot < 0 || slot >= (int)b->ctx.size() || !b->ctx[(size_t)slot])
        return fail(PIC_ERR_INVALID_ARG, "no discharge in this slot");
    CK(cudaStreamSynchronize(b->stream));
    pic_destroy(b->ctx[(size_t)slot]);
    CK(cudaFree(b->phase[(size_t)slot]));
    b->ctx[(size_t)slot] = nullptr;
    b->phase[(size_t)slot] = nullptr;
    b->dirty = true;
    return PIC_OK;
}

int pic_batch_ctx(pic_batch* b, int slot, pic_ctx** out)
{
    if (!b || !out || slot < 0 || slot >= (int)b->ctx.size() || !b->ctx[(size_t)slot])
        return fail(PIC_ERR_INVALID_ARG, "no discharge in this slot");
    *out = b->ctx[(size_t)slot];
    return PIC_OK;
}

int pic_batch_set_chunk(pic_batch* b, int64_t particles_per_chunk)
{
    if (!b || particles_per_chunk < 0) return fail(PIC_ERR_INVALID_ARG, "bad batch or chunk size");
    CK(cudaStreamSynchronize(b->stream));
    b->chunk = particles_per_chunk;
    b->dirty = true;
    return PIC_OK;
}

int pic_batch_set_target(pic_batch* b, int64_t particles_per_cta)
{
    if (!b || (particles_per_cta != 0 && particles_per_cta < 1024))
        return fail(PIC_ERR_INVALID_ARG, "particles per CTA: 0 (automatic) or >= 1024");
    b->target = particles_per_cta;
    b->dirty = true;
    return PIC_OK;
}

int pic_batch_step(pic_batch* b, int64_t n)
{
    if (!b || n < 0) return fail(PIC_ERR_INVALID_ARG, "bad batch or step count");
    if (n == 0) return PIC_OK;
    pic_ctx* first = nullptr;
    for (pic_ctx* c : b->ctx) {
        if (!c) continue;
        if (!first) first = c;
        const int de = c->p.diag_every;
        if (de > 0 && c->h_step % de != first->h_step % de)
            return fail(PIC_ERR_INVALID_ARG, "batch members out of step with the sampling period");
    }
    if (!first) return PIC_OK;
    if (b->dirty) {
        int rc = batch_rebuild(b);
        if (rc) return rc;
    }
    // the first step of this call enters the averages unless a field call already added it
    size_t e = 0;
    for (pic_ctx* c : b->ctx) {
        if (!c) continue;
        b->h_ent[e].d = c->d;
        b->h_ent[e].acc_from = (unsigned int)(c->acc_upto + 1);
        ++e;
    }
    CK(cudaMemcpyAsync(b->d_ent, b->h_ent.data(), b->h_ent.size() * sizeof(BatchEntry), cudaMemcpyHostToDevice,
                       b->stream));
    const int de = first->p.diag_every;
    int64_t k = 0;
    while (k < n) {
        const long long l = first->h_step;
        const bool block = b->use_graph && de > 1 && l % de == 0 && n - k >= de && !batch_sort_inside(b, l, de);
        if (block && !b->gexec) {
            int rc = batch_capture(b, de);
            if (rc) return rc;
        }
        int rc = batch_timer(b, block ? de : 1, true);
        if (rc) return rc;
        if (block) CK(cudaGraphLaunch(b->gexec, b->stream));
        else CK(batch_launch(b, de > 0 && (l + 1) % de == 0, b->stream));
        rc = batch_timer(b, 0, false);
        if (rc) return rc;
        const int m = block ? de : 1;
        for (int j = 0; j < m; ++j) {
            rc = batch_advance(b);
            if (rc) return rc;
        }
        k += m;
    }
    return PIC_OK;
}

int pic_batch_graphs(pic_batch* b, int enable)
{
    if (!b) return fail(PIC_ERR_INVALID_ARG, "batch is NULL");
    b->use_graph = enable != 0;
    return PIC_OK;
}

int pic_batch_timing(pic_batch* b, int enable, double* ms, int64_t* steps)
{
    if (!b) return fail(PIC_ERR_INVALID_ARG, "batch is NULL");
    CK(cudaStreamSynchronize(b->stream));
    int rc = batch_timers_collect(b);
    if (rc) return rc;
    if (ms) *ms = b->t_ms;
    if (steps) *steps = b->t_steps;
    b->t_ms = 0.0;
    b->t_steps = 0;
    b->timing = enable != 0;
    return PIC_OK;
}

int pic_batch_autotune(pic_batch* b, const int64_t* candidates, int n_cand, int64_t steps_each, int64_t* best)
{
    static const int64_t kDefault[] = {8192, 16384, 32768, 65536, 131072, 262144};
    if (!b || n_cand < 0 || steps_each < 1) return fail(PIC_ERR_INVALID_ARG, "bad autotune arguments");
    if (!candidates || n_cand == 0) {
        candidates = kDefault;
        n_cand = (int)(sizeof(kDefault) / sizeof(kDefault[0]));
    }
    const bool was = b->timing;
    double best_ms = 0.0;
    int64_t best_t = b->target;
    for (int i = 0; i < n_cand; ++i) {
        int rc = pic_batch_set_target(b, candidates[i]);
        if (rc) return rc;
        rc = pic_batch_step(b, 1);                       // rebuild and first launch outside the window
        if (rc) return rc;
        rc = pic_batch_timing(b, 1, nullptr, nullptr);
        if (rc) return rc;
        rc = pic_batch_step(b, steps_each);
        if (rc) return rc;
        double ms = 0.0;
        int64_t st = 0;
        rc = pic_batch_timing(b, was, &ms, &st);
        if (rc) return rc;
        const double per = st > 0 ? ms / (double)st : 0.0;
        if (i == 0 || per < best_ms) {
            best_ms = per;
            best_t = candidates[i];
        }
    }
    int rc = pic_batch_set_target(b, best_t);
    if (rc) return rc;
    if (best) *best = best_t;
    return PIC_OK;
}

int pic_batch_sync(pic_batch* b)
{
    if (!b) return fail(PIC_ERR_INVALID_ARG, "batch is NULL");
    for (pic_ctx* c : b->ctx) {
        if (!c) continue;
        int rc = pic_sync(c);
        if (rc) return rc;
    }
    return PIC_OK;
}

void pic_batch_destroy(pic_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    for (size_t k = 0; k < b->ctx.size(); ++k) {
        if (b->ctx[k]) pic_destroy(b->ctx[k]);
        if (b->phase[k]) cudaFree(b->phase[k]);
    }
    if (b->d_ent) cudaFree(b->d_ent);
    if (b->d_owner) cudaFree(b->d_owner);
    if (b->d_chunk) cudaFree(b->d_chunk);
    if (b->d_work) cudaFree(b->d_work);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (cudaEvent_t ev : b->tev) cudaEventDestroy(ev);
    delete b;
}

}  // extern "C"
