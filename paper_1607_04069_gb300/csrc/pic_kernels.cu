// pic_kernels.cu -- PIC/MCC kernels for sm_103a.
//
// k_mover is the hot path: one launch per time step moves every charged
// superparticle through one cycle of the paper's Fig. 4 loop (field
// interpolation -> leapfrog push -> wall interaction -> null-collision MCC)
// and deposits x^{l+1} into per-CTA int64 shared-memory histograms; the last
// CTA to finish solves Poisson's equation for step l+1 (solve.cuh).
#include <type_traits>

#include "common.cuh"
#include "launch.h"
#include "solve.cuh"

namespace pg {

// ---------------------------------------------------------------- init
// Initial loading (Sec. "Kinetic Particle Simulation"): uniform positions,
// Maxwellian velocities at T (eV) by Box-Muller, ids tag | k.
template <bool P64>
__global__ void k_init(Dev d, int s, long long n, float vth)
{
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const SpBuf B = d.buf[s][d.ctl->cur[s]];
    const uint64_t id = id_tag(s) | (uint64_t)k;
    const uint4 a = draw(d.seed, id, 0, kPurInit);
    const uint4 b = draw(d.seed, id, 1, kPurInit);
    const uint32_t fx = a.x | 1u;
    if (P64) ((double*)B.pos)[k] = (double)d.ncell * ((double)fx * 0x1p-32);
    else ((uint32_t*)B.pos)[k] = fx;
    const float2 n12 = box_muller(a.y, a.z);
    const float2 n34 = box_muller(b.x, b.y);
    B.vx[k] = vth * n12.x;
    B.vy[k] = vth * n12.y;
    B.vz[k] = vth * n34.x;
    B.id[k] = id;
}

// ---------------------------------------------------------------- helpers
struct BlockTally {            // per-CTA event counts, flushed once per CTA
    unsigned int elastic, excit, ioniz, cx, iso, numerics, capacity;
};

__device__ __forceinline__ void hist_add(unsigned long long* h, int nb, float x, float xmax)
{
    int b = (int)(x / xmax * (float)nb);
    b = b < 0 ? 0 : (b > nb - 1 ? nb - 1 : b);
    atomicAdd(&h[b], 1ull);
}

// Wall interaction of an Ar+ (Sec. "Wall Interaction"): energy and angle into
// the IEDF / IEADF, then sputtered-atom launch (Sec. "Wall Interactions" of the
// TPM: N = ceil(Y) trials with R <= Y/N, Thompson energy, cosine angle).
__device__ void ion_wall(const Dev& d, uint64_t id, uint32_t l, int el, float vx, float vy, float vz,
                         long long n_tp0, BlockTally* tally)
{
    const float v2 = vx * vx + vy * vy + vz * vz;
    const float E = v2 * (float)(0.5 * kMAR / kQE);
    float ct = v2 > 0.0f ? fabsf(vx) * rsqrtf(v2) : 1.0f;
    ct = fminf(ct, 1.0f);
    const float th = acosf(ct) * (float)(180.0 / kPI);
    hist_add(d.diag.iedf[el], kNbIedf, E, d.Emax_hist);
    int be = (int)(E / d.Emax_hist * (float)kNbIeadfE);
    be = be < 0 ? 0 : (be > kNbIeadfE - 1 ? kNbIeadfE - 1 : be);
    int ba = (int)th;
    ba = ba < 0 ? 0 : (ba > kNbAng - 1 ? kNbAng - 1 : ba);
    atomicAdd(&d.diag.ieadf[el][be * kNbAng + ba], 1ull);
    atomicAdd(&d.ctl->cnt[el == 0 ? kCntImpIL : kCntImpIR], 1ull);
    if (!d.sputter || !(E > (float)kSpTh)) return;
    const float Y = 0.1f * sqrtf(E / (float)kSpTh - 1.0f);
    int Nt = (int)ceilf(Y);
    Nt = Nt > kSpMaxN ? kSpMaxN : Nt;
    const float Emax = lambda_ar_al() * E;
    const SpBuf T = d.buf[kTP][d.ctl->cur[kTP]];
    uint4 t = make_uint4(0, 0, 0, 0);
    for (int k = 0; k < Nt; ++k) {
        if ((k & 3) == 0) t = draw(d.seed, id, l, kPurSpTrial + (k >> 2));
        const uint32_t w = (k & 3) == 0 ? t.x : (k & 3) == 1 ? t.y : (k & 3) == 2 ? t.z : t.w;
        if (!(u23(w) <= Y / (float)Nt)) continue;
        const uint4 ce = draw(d.seed, id, l, kPurSpEmit + k);
        const uint4 ci = draw(d.seed, id, l, kPurSpId + k);
        const float3 v = emit(u23(ce.x), u23(ce.y), u23(ce.z), Emax, el == 0 ? 1.0f : -1.0f);
        const long long idx = n_tp0 + atomicAdd((unsigned long long*)&d.ctl->births[kTP], 1ull);
        if (idx >= d.ctl->cap[kTP]) {
            atomicAdd(&tally->capacity, 1u);
            continue;
        }
        ((uint32_t*)T.pos)[idx] = el == 0 ? 1u : 0xffffffffu;
        T.vx[idx] = v.x;
        T.vy[idx] = v.y;
        T.vz[idx] = v.z;
        T.id[idx] = child_id(ci.x, ci.y, kTP);
        atomicAdd(&d.ctl->cnt[el == 0 ? kCntSputL : kCntSputR], 1ull);
    }
}

template <typename PosT>
__device__ __forceinline__ void store_dead(PosT* P, long long i);
template <>
__device__ __forceinline__ void store_dead<uint32_t>(uint32_t* P, long long i) { P[i] = 0u; }
template <>
__device__ __forceinline__ void store_dead<double>(double* P, long long i) { P[i] = -1.0; }

// Electron null-collision MCC (Sec. "Particle Collisions"): process chosen by
// R nu_max against the cumulative nu_el, nu_exc, nu_ion at the electron's
// energy; elastic and excitation scatter isotropically, ionisation splits the
// remaining energy uniformly and creates an e-/Ar+ pair at x^{l+1}.
template <typename PosT>
__device__ void mcc_electron(const Dev& d, uint4 c, uint64_t id, uint32_t l, PosT xn, float& vx,
                             float& vy, float& vz, long long n0e, long long n0i,
                             unsigned long long* sq, BlockTally* tally)
{
    const float v2 = vx * vx + vy * vy + vz * vz;
    const float v = sqrtf(v2);
    const float eps = v2 * (float)(0.5 * kME / kQE);
    if (eps > d.eps_max) atomicAdd(&tally->numerics, 1u);
    const float s_exc = eps > (float)kExcTh ? (float)kExcSig * (1.0f - (float)kExcTh / eps) : 0.0f;
    const float s_ion = eps > (float)kIonTh
                            ? (float)(kLotzA * kLotzQ) * logf(eps / (float)kIonTh) / (eps * (float)kIonTh)
                            : 0.0f;
    const float nu_el = d.ngas_f * (float)kSigEl * v;
    const float nu_exc = d.ngas_f * s_exc * v;
    const float nu_ion = d.ngas_f * s_ion * v;
    const float r = u23(c.y) * d.nu_max_e;
    const float3 dir = iso_dir(c.z, c.w);
    if (r < nu_el) {
        const float cchi = v > 0.0f ? (dir.x * vx + dir.y * vy + dir.z * vz) / v : 1.0f;
        const float fac = 1.0f - (float)(2.0 * kME / kMAR) * (1.0f - cchi);
        const float vn = v * sqrtf(fac);
        vx = vn * dir.x; vy = vn * dir.y; vz = vn * dir.z;
        atomicAdd(&tally->elastic, 1u);
    } else if (r < nu_el + nu_exc) {
        const float vn = sqrtf((eps - (float)kExcTh) * (float)(2.0 * kQE / kME));
        vx = vn * dir.x; vy = vn * dir.y; vz = vn * dir.z;
        atomicAdd(&tally->excit, 1u);
    } else if (r < nu_el + nu_exc + nu_ion) {
        const float epr = eps - (float)kIonTh;
        const uint4 ci = draw(d.seed, id, l, kPurIonize);
        const uint4 cn = draw(d.seed, id, l, kPurNewIon);
        const uint4 cb = draw(d.seed, id, l, kPurBirthId);
        const float e_ej = u23(ci.x) * epr;
        const float e_sc = epr - e_ej;
        const float vs = sqrtf(e_sc * (float)(2.0 * kQE / kME));
        const float ve = sqrtf(e_ej * (float)(2.0 * kQE / kME));
        const float3 d2 = iso_dir(ci.y, ci.z);
        const float2 n12 = box_muller(cn.x, cn.y);
        const float2 n34 = box_muller(cn.z, cn.w);
        vx = vs * dir.x; vy = vs * dir.y; vz = vs * dir.z;
        atomicAdd(&tally->ioniz, 1u);
        const long long ie = n0e + atomicAdd((unsigned long long*)&d.ctl->births[kE], 1ull);
        const long long ii = n0i + atomicAdd((unsigned long long*)&d.ctl->births[kI], 1ull);
        const bool ok = ie < d.ctl->cap[kE] && ii < d.ctl->cap[kI];
        const SpBuf Be = d.buf[kE][d.ctl->cur[kE]];
        const SpBuf Bi = d.buf[kI][d.ctl->cur[kI]];
        if (!ok) {
            atomicAdd(&tally->capacity, 1u);
            if (ie < d.ctl->cap[kE]) store_dead((PosT*)Be.pos, ie);
            if (ii < d.ctl->cap[kI]) store_dead((PosT*)Bi.pos, ii);
            return;
        }
        ((PosT*)Be.pos)[ie] = xn;
        Be.vx[ie] = ve * d2.x; Be.vy[ie] = ve * d2.y; Be.vz[ie] = ve * d2.z;
        Be.id[ie] = child_id(cb.x, cb.y, kE);
        ((PosT*)Bi.pos)[ii] = xn;
        Bi.vx[ii] = d.vth_gas * n12.x; Bi.vy[ii] = d.vth_gas * n12.y; Bi.vz[ii] = d.vth_gas * n34.x;
        Bi.id[ii] = child_id(cb.z, cb.w, kI);
        uint32_t j, wr;
        cell_of(xn, d.kshift, j, wr);
        atomicAdd(&sq[j], (1ull << 32) - wr);                 // electron child: this CTA's histogram
        if (wr) atomicAdd(&sq[j + 1], (unsigned long long)wr);
        atomicAdd(&d.q[kI][j], (1ull << 32) - wr);            // ion child: global histogram
        if (wr) atomicAdd(&d.q[kI][j + 1], (unsigned long long)wr);
    }
}

// Ar+ null-collision MCC against a Maxwellian gas partner.  sigma(eps) g is
// the same constant for both channels, so the selection R nu_max < nu_cx
// reduces exactly to R < 1/2 (R sits on the 2^-23 grid + 1/2, never at 1/2).
__device__ __forceinline__ void mcc_ion(const Dev& d, uint4 c, uint64_t id, uint32_t l, float& vx,
                                        float& vy, float& vz, BlockTally* tally)
{
    const uint4 cg = draw(d.seed, id, l, kPurGas);
    const float2 n12 = box_muller(cg.x, cg.y);
    const float2 n34 = box_muller(cg.z, cg.w);
    const float wx = d.vth_gas * n12.x, wy = d.vth_gas * n12.y, wz = d.vth_gas * n34.x;
    if (u23(c.y) < 0.5f) {
        vx = wx; vy = wy; vz = wz;
        atomicAdd(&tally->cx, 1u);
    } else {
        const float gx = vx - wx, gy = vy - wy, gz = vz - wz;
        const float gm = sqrtf(gx * gx + gy * gy + gz * gz);
        const float3 dir = iso_dir(c.z, c.w);
        vx = 0.5f * (vx + wx) + 0.5f * gm * dir.x;
        vy = 0.5f * (vy + wy) + 0.5f * gm * dir.y;
        vz = 0.5f * (vz + wz) + 0.5f * gm * dir.z;
        atomicAdd(&tally->iso, 1u);
    }
}

// split of the grid between the two species, proportional to their counts
__device__ __forceinline__ int electron_ctas(long long ne, long long ni, int G)
{
    if (ne <= 0) return 0;
    if (ni <= 0) return G;
    int Ge = (int)((double)G * (double)ne / (double)(ne + ni) + 0.5);
    return Ge < 1 ? 1 : (Ge > G - 1 ? G - 1 : Ge);
}

__device__ __forceinline__ void flush_tally(const Dev& d, const BlockTally& t)
{
    Ctl* c = d.ctl;
    if (t.elastic) atomicAdd(&c->cnt[kCntElastic], (unsigned long long)t.elastic);
    if (t.excit) atomicAdd(&c->cnt[kCntExcit], (unsigned long long)t.excit);
    if (t.ioniz) atomicAdd(&c->cnt[kCntIoniz], (unsigned long long)t.ioniz);
    if (t.cx) atomicAdd(&c->cnt[kCntCx], (unsigned long long)t.cx);
    if (t.iso) atomicAdd(&c->cnt[kCntIso], (unsigned long long)t.iso);
    if (t.numerics) {
        atomicAdd(&c->cnt[kCntNumerics], (unsigned long long)t.numerics);
        atomicOr(&c->err, kErrNumerics);
    }
    if (t.capacity) {
        atomicAdd(&c->cnt[kCntCapacity], (unsigned long long)t.capacity);
        atomicOr(&c->err, kErrCapacity);
    }
}

// ---------------------------------------------------------------- mover
// MODE 0: full PIC/MCC step.  MODE 1: deposit the current state and solve
// for the field at the current step (creation, after a state upload).
template <bool P64, int MODE>
__global__ void __launch_bounds__(kMoverThreads) k_mover(Dev d)
{
    using PosT = typename std::conditional<P64, double, uint32_t>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N1 = d.ncell + 1;
    unsigned long long* sq = (unsigned long long*)smem_raw;
    long long* sflux = (long long*)(sq + N1);
    float* sE = (float*)(sflux + N1);
    unsigned int* seedf = (unsigned int*)(sE + ((N1 + 3) & ~3));
    __shared__ BlockTally tally;
    __shared__ unsigned int s_jlo, s_jhi;
    __shared__ int s_last;

    Ctl* ctl = d.ctl;
    const unsigned int l = ctl->step;
    const long long ne = ctl->n[kE], ni = ctl->n[kI], ntp = ctl->n[kTP];
    const bool sample = MODE == 0 && d.diag_every > 0 && ((l + 1) % (unsigned)d.diag_every == 0);
    const int G = gridDim.x;
    const int Ge = electron_ctas(ne, ni, G);
    const int s = (int)blockIdx.x < Ge ? kE : kI;
    const int b = s == kE ? blockIdx.x : blockIdx.x - Ge;
    const int Gs = s == kE ? Ge : G - Ge;
    const long long ns = s == kE ? ne : ni;
    const long long beg = ns * b / Gs, end = ns * (b + 1) / Gs;

    for (int i = threadIdx.x; i < N1; i += blockDim.x) {
        sq[i] = 0;
        sflux[i] = 0;
        sE[i] = d.E32[i];
    }
    for (int i = threadIdx.x; i < kNbEedf; i += blockDim.x) seedf[i] = 0;
    if (threadIdx.x == 0) {
        tally = BlockTally{0, 0, 0, 0, 0, 0, 0};
        s_jlo = 0xffffffffu;
        s_jhi = 0;
    }
    __syncthreads();

    const SpBuf B = d.buf[s][ctl->cur[s]];
    PosT* __restrict__ P = (PosT*)B.pos;
    float* __restrict__ VX = B.vx;
    const uint64_t* __restrict__ ID = B.id;
    const float qmdt = d.qm_dt[s];
    const unsigned long long thr = d.thr[s];
    uint32_t jlo = 0xffffffffu, jhi = 0;

    for (long long i0 = beg; i0 < end; i0 += blockDim.x) {
        const long long i = i0 + threadIdx.x;
        bool act = i < end;
        PosT x = 0;
        float vx = 0.0f;
        if (act) {
            x = P[i];
            act = is_alive(x);
            if (P64 && act && !((double)x < (double)d.ncell)) {
                act = false;
                atomicOr(&ctl->err, kErrIndex);
            }
        }
        uint32_t j = 0, wr = 0;
        bool dep = false;
        if (act) {
            if (MODE == 1) {
                cell_of(x, d.kshift, j, wr);
                dep = true;
            } else {
                vx = VX[i];
                const uint64_t id = ID[i];
                // field interpolation: the same linear weights as the deposit
                uint32_t jj, ww;
                cell_of(x, d.kshift, jj, ww);
                const float f = (float)ww * 0x1p-32f;
                const float Ex = (1.0f - f) * sE[jj] + f * sE[jj + 1];
                // leapfrog: v^{l+1/2} = v^{l-1/2} + (q/m) E dt ; x^{l+1} = x^l + v dt
                vx = vx + qmdt * Ex;
                PosT xn;
                bool out;
                int el;
                if (P64) {
                    const double xd = (double)x + (double)vx * d.push64;
                    out = xd <= 0.0 || xd >= (double)d.ncell;
                    el = xd <= 0.0 ? 0 : 1;
                    xn = (PosT)xd;
                } else {
                    const long long np = (long long)x + __float2ll_rn(vx * d.push32);
                    out = np <= 0 || np >= 4294967296LL;
                    el = np <= 0 ? 0 : 1;
                    xn = (PosT)(unsigned long long)np;
                }
                if (out) {
                    store_dead(P, i);
                    if (s == kI)
                        ion_wall(d, id, l, el, vx, B.vy[i], B.vz[i], ntp, &tally);
                    else
                        atomicAdd(&ctl->cnt[el == 0 ? kCntImpEL : kCntImpER], 1ull);
                } else {
                    const uint4 c = draw(d.seed, id, l, kPurColl);
                    if ((unsigned long long)c.x < thr) {
                        float vy = B.vy[i], vz = B.vz[i];
                        if (s == kE)
                            mcc_electron<PosT>(d, c, id, l, xn, vx, vy, vz, ne, ni, sq, &tally);
                        else
                            mcc_ion(d, c, id, l, vx, vy, vz, &tally);
                        B.vy[i] = vy;
                        B.vz[i] = vz;
                    }
                    P[i] = xn;
                    VX[i] = vx;
                    cell_of(xn, d.kshift, j, wr);
                    dep = true;
                    if (sample) {
                        const long long vq = (long long)__float2int_rn(vx);
                        atomicAdd((unsigned long long*)&sflux[j],
                                  (unsigned long long)(vq * (long long)(((1ull << 32) - wr) >> 16)));
                        atomicAdd((unsigned long long*)&sflux[j + 1],
                                  (unsigned long long)(vq * (long long)(wr >> 16)));
                        if (s == kE) {
                            bool inwin;
                            if (P64) inwin = (double)xn >= d.eedf_lo64 && (double)xn < d.eedf_hi64;
                            else inwin = (uint32_t)xn >= d.eedf_lo && (uint32_t)xn < d.eedf_hi;
                            if (inwin) {
                                const float vy = B.vy[i], vz = B.vz[i];
                                const float e = (vx * vx + vy * vy + vz * vz) * (float)(0.5 * kME / kQE);
                                int bb = (int)(e * 4.0f);
                                bb = bb < 0 ? 0 : (bb > kNbEedf - 1 ? kNbEedf - 1 : bb);
                                atomicAdd(&seedf[bb], 1u);
                            }
                        }
                    }
                }
            }
        }
        if (dep) {
            jlo = min(jlo, j);
            jhi = max(jhi, j);
        }
        warp_deposit(sq, dep, j, wr);
    }
    // range of touched nodes (newborns sit in cells their parents touched)
    jlo = __reduce_min_sync(0xffffffffu, jlo);
    jhi = __reduce_max_sync(0xffffffffu, jhi);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&s_jlo, jlo);
        atomicMax(&s_jhi, jhi);
    }
    __syncthreads();
    if (s_jlo != 0xffffffffu) {
        for (int m = (int)s_jlo + threadIdx.x; m <= (int)s_jhi + 1; m += blockDim.x) {
            const unsigned long long v = sq[m];
            if (v) atomicAdd(&d.q[s][m], v);
            if (sample) {
                const long long f = sflux[m];
                if (f) atomicAdd((unsigned long long*)&d.flux[s][m], (unsigned long long)f);
            }
        }
    }
    if (sample && s == kE)
        for (int i = threadIdx.x; i < kNbEedf; i += blockDim.x)
            if (seedf[i]) atomicAdd(&d.diag.eedf[i], (unsigned long long)seedf[i]);
    if (threadIdx.x == 0) flush_tally(d, tally);
    // last CTA: field solve for the new step
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ctl->done, 1u) == (unsigned)(G - 1);
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (MODE == 0) finish_step(d, l + 1, true, sample);
        else finish_step(d, l, false, false);
    }
}

// ---------------------------------------------------------------- standalone ops
template <typename PosT>
__global__ void __launch_bounds__(kMoverThreads)
    k_op_deposit(const PosT* __restrict__ pos, long long n, int ncell, int kshift,
                 unsigned long long* q)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long* sq = (unsigned long long*)smem_raw;
    const int N1 = ncell + 1;
    for (int i = threadIdx.x; i < N1; i += blockDim.x) sq[i] = 0;
    __syncthreads();
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long beg = per * blockIdx.x, end = min(n, beg + per);
    for (long long i0 = beg; i0 < end; i0 += blockDim.x) {
        const long long i = i0 + threadIdx.x;
        bool act = i < end;
        PosT x = 0;
        if (act) {
            x = pos[i];
            act = is_alive(x);
        }
        uint32_t j = 0, wr = 0;
        if (act) {
            cell_of(x, kshift, j, wr);
            if (j >= (uint32_t)ncell) act = false;
        }
        warp_deposit(sq, act, j, wr);
    }
    __syncthreads();
    for (int m = threadIdx.x; m < N1; m += blockDim.x)
        if (sq[m]) atomicAdd(&q[m], sq[m]);
}

__global__ void k_op_poisson(const long long* qi, const long long* qe, int N, double A, double inv_dx,
                             double v_left, double* phi, double* E64)
{
    QNet qn{(const unsigned long long*)qi, (const unsigned long long*)qe, false};
    poisson_block(qn, N, A, inv_dx, v_left, phi, E64, nullptr);
}

// ---------------------------------------------------------------- sort / compaction
// Counting sort by cell of one species into the other ping-pong half; removed
// particles are dropped and the births of earlier steps are merged in.
template <typename PosT>
__global__ void k_sort_count(Dev d, int s)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned int* sc = (unsigned int*)smem_raw;
    const int N = d.ncell;
    for (int i = threadIdx.x; i < N; i += blockDim.x) sc[i] = 0;
    __syncthreads();
    const long long n = d.ctl->n[s];
    const PosT* P = (const PosT*)d.buf[s][d.ctl->cur[s]].pos;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const PosT x = P[i];
        if (!is_alive(x)) continue;
        uint32_t j, wr;
        cell_of(x, d.kshift, j, wr);
        if (j >= (uint32_t)N) continue;
        atomicAdd(&sc[j], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        if (sc[i]) atomicAdd(&d.sort_cnt[i], sc[i]);
}

__global__ void k_sort_scan(Dev d)
{
    __shared__ long long sh[32];
    const int N = d.ncell, T = blockDim.x, t = threadIdx.x;
    const int seg = (N + T - 1) / T;
    const int m0 = min(t * seg, N), m1 = min(m0 + seg, N);
    long long a = 0;
    for (int m = m0; m < m1; ++m) a += d.sort_cnt[m];
    long long tot;
    long long off = block_exclusive_scan(a, sh, tot);
    for (int m = m0; m < m1; ++m) {
        const unsigned int c = d.sort_cnt[m];
        d.sort_off[m] = (unsigned int)off;
        off += c;
        d.sort_cnt[m] = 0;
    }
    if (t == 0) d.ctl->sort_total = tot;
}

template <typename PosT>
__global__ void k_sort_scatter(Dev d, int s)
{
    __shared__ int s_last;
    const long long n = d.ctl->n[s];
    const unsigned int cur = d.ctl->cur[s];
    const SpBuf A = d.buf[s][cur], Bn = d.buf[s][cur ^ 1u];
    const PosT* PA = (const PosT*)A.pos;
    PosT* PB = (PosT*)Bn.pos;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long nround = (n + stride - 1) / stride * stride;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nround; i += stride) {
        bool act = i < n;
        PosT x = 0;
        if (act) {
            x = PA[i];
            act = is_alive(x);
        }
        uint32_t j = 0xffffffffu, wr;
        if (act) {
            cell_of(x, d.kshift, j, wr);
            if (j >= (uint32_t)d.ncell) {
                act = false;
                j = 0xffffffffu;
            }
        }
        const unsigned grp = __match_any_sync(0xffffffffu, j);
        const int leader = __ffs(grp) - 1;
        const int rank = __popc(grp & ((1u << lane) - 1u));
        unsigned int base = 0;
        if (act && lane == leader) base = atomicAdd(&d.sort_off[j], (unsigned)__popc(grp));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (act) {
            const unsigned int o = base + rank;
            PB[o] = x;
            Bn.vx[o] = A.vx[i];
            Bn.vy[o] = A.vy[i];
            Bn.vz[o] = A.vz[i];
            Bn.id[o] = A.id[i];
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&d.ctl->sort_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        d.ctl->n[s] = d.ctl->sort_total;
        d.ctl->cur[s] = cur ^ 1u;
        d.ctl->sort_done = 0;
    }
}

// ---------------------------------------------------------------- launchers
size_t mover_smem(int ncell)
{
    const int N1 = ncell + 1;
    return (size_t)N1 * 16 + (size_t)((N1 + 3) & ~3) * 4 + kNbEedf * 4;
}

cudaError_t launch_init(const Dev& d, int s, long long n, float vth, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int T = 256;
    const long long G = (n + T - 1) / T;
    if (d.pos64 && s != kTP) k_init<true><<<(unsigned)G, T, 0, st>>>(d, s, n, vth);
    else k_init<false><<<(unsigned)G, T, 0, st>>>(d, s, n, vth);
    return cudaGetLastError();
}

static cudaError_t set_smem_attr(const void* fn, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_mover(const Dev& d, int grid, int mode, cudaStream_t st)
{
    const size_t sm = mover_smem(d.ncell);
    const void* fn;
    if (d.pos64) fn = mode == 0 ? (const void*)k_mover<true, 0> : (const void*)k_mover<true, 1>;
    else fn = mode == 0 ? (const void*)k_mover<false, 0> : (const void*)k_mover<false, 1>;
    cudaError_t e = set_smem_attr(fn, sm);
    if (e != cudaSuccess) return e;
    if (d.pos64) {
        if (mode == 0) k_mover<true, 0><<<grid, kMoverThreads, sm, st>>>(d);
        else k_mover<true, 1><<<grid, kMoverThreads, sm, st>>>(d);
    } else {
        if (mode == 0) k_mover<false, 0><<<grid, kMoverThreads, sm, st>>>(d);
        else k_mover<false, 1><<<grid, kMoverThreads, sm, st>>>(d);
    }
    return cudaGetLastError();
}

cudaError_t launch_sort(const Dev& d, int s, int grid, cudaStream_t st)
{
    const bool p64 = d.pos64 && s != kTP;
    const size_t sm = (size_t)d.ncell * 4;
    if (p64) k_sort_count<double><<<grid, 256, sm, st>>>(d, s);
    else k_sort_count<uint32_t><<<grid, 256, sm, st>>>(d, s);
    k_sort_scan<<<1, 1024, 0, st>>>(d);
    if (p64) k_sort_scatter<double><<<grid, 256, 0, st>>>(d, s);
    else k_sort_scatter<uint32_t><<<grid, 256, 0, st>>>(d, s);
    return cudaGetLastError();
}

cudaError_t launch_op_deposit(const void* pos, int pos64, long long n, int ncell, int kshift,
                              unsigned long long* q, int grid, cudaStream_t st)
{
    const size_t sm = (size_t)(ncell + 1) * 8;
    if (pos64) {
        cudaError_t e = set_smem_attr((const void*)k_op_deposit<double>, sm);
        if (e != cudaSuccess) return e;
        k_op_deposit<double><<<grid, kMoverThreads, sm, st>>>((const double*)pos, n, ncell, kshift, q);
    } else {
        cudaError_t e = set_smem_attr((const void*)k_op_deposit<uint32_t>, sm);
        if (e != cudaSuccess) return e;
        k_op_deposit<uint32_t><<<grid, kMoverThreads, sm, st>>>((const uint32_t*)pos, n, ncell, kshift, q);
    }
    return cudaGetLastError();
}

cudaError_t launch_op_poisson(const long long* qi, const long long* qe, int N, double A, double inv_dx,
                              double v_left, double* phi, double* E64, cudaStream_t st)
{
    k_op_poisson<<<1, 512, 0, st>>>(qi, qe, N, A, inv_dx, v_left, phi, E64);
    return cudaGetLastError();
}

}  // namespace pg
