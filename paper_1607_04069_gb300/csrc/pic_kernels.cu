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
__global__ void k_init(Dev d, int s, long long n, long long id0, float vth)
{
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const SpBuf B = d.buf[s][d.ctl->cur[s]];
    const uint64_t id = id_tag(s) | (uint64_t)(id0 + k);
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
    if (s != kTP) B.nev[k] = entry_nev(d, s, id, 0);
}

// ---------------------------------------------------------------- helpers
struct BlockTally {            // per-CTA event counts, flushed once per CTA
    unsigned int elastic, excit, ioniz, cx, iso, numerics, capacity;
    unsigned int imp_e[2], imp_i[2], sput[2];
};

__device__ __forceinline__ void hist_add(unsigned long long* h, int nb, float x, float xmax)
{
    atomicAdd(&h[hist_bin(x, xmax, nb)], 1ull);
}

// value that marks a removed slot
template <typename PosT> __device__ __forceinline__ PosT dead_value();
template <> __device__ __forceinline__ uint32_t dead_value<uint32_t>() { return 0u; }
template <> __device__ __forceinline__ double dead_value<double>() { return -1.0; }

// ---------------------------------------------------------------- events
// An event is a dependent chain, and the last events of a CTA decide when it
// ends.  Each event therefore draws its Philox blocks two at a time
// (interleaved rounds) and keeps the frequent work inline, while rare
// outcomes -- an ionisation, an Ar+ collision or wall hit, the FP64 branch of
// a candidate gap -- run out of line and call the shared out-of-line draws,
// directions and samples.  Those stay in the instruction cache because the
// frequent events use them, so a rare outcome fetches little code of its
// own; inlined, each rare path would be a separate body of code that is cold
// whenever it runs.
struct U4x2 {
    uint4 a, b;
};
// two Philox blocks under the seed's key with interleaved rounds
__device__ __noinline__ U4x2 ev_draw2(uint64_t seed, uint64_t ida, uint32_t stepa, uint32_t pa, uint64_t idb,
                                      uint32_t stepb, uint32_t pb)
{
    uint4 c[2];
    c[0] = make_uint4((uint32_t)ida, (uint32_t)(ida >> 32), stepa, pa);
    c[1] = make_uint4((uint32_t)idb, (uint32_t)(idb >> 32), stepb, pb);
    philox_n<2>(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    return U4x2{c[0], c[1]};
}
__device__ __noinline__ float3 ev_iso_dir(uint32_t a, uint32_t b) { return iso_dir(a, b); }
__device__ __noinline__ float2 ev_box_muller(uint32_t a, uint32_t b) { return box_muller(a, b); }
__device__ __noinline__ uint32_t ev_gap_exact(double lam, uint32_t w) { return gap_exact(lam, w); }
__device__ __forceinline__ uint32_t ev_gap(double lam, float lamf, uint32_t w)
{
    uint32_t g;
    return gap_fast(lamf, w, g) ? g : ev_gap_exact(lam, w);
}
// tabulated cross section (Sec. "Particle Collisions": look-up tables):
// linear between the points, constant beyond the first and the last
__device__ __noinline__ float ev_xs_table(const float2* t, int n, float eps)
{
    if (eps <= t[0].x) return t[0].y;
    if (eps >= t[n - 1].x) return t[n - 1].y;
    int lo = 0, hi = n - 1;                       // t[lo].x <= eps < t[hi].x
    while (hi - lo > 1) {
        const int mid = lo + (hi - lo) / 2;
        if (t[mid].x <= eps) lo = mid;
        else hi = mid;
    }
    const float2 a = t[lo], b = t[hi];
    return a.y + (eps - a.x) / (b.x - a.x) * (b.y - a.y);
}
__device__ __noinline__ float3 ev_emit(float uE, float uT, float uP, float Emax, float dir)
{
    return emit(uE, uT, uP, Emax, dir);
}

// Ionisation (Sec. "Particle Collisions"): the remaining energy eps - 15.8 eV
// is split uniformly between the scattered and the ejected electron (ci: the
// IONIZE words), and an e-/Ar+ pair is born at x^{l+1}, the ion from the gas
// Maxwellian, each child with its first candidate step (births are pushed
// from step l+1 on).  The slots are reserved first: their atomics are the
// longest wait and overlap the draws.  Returns the scattered electron's speed.
template <typename PosT>
__device__ __noinline__ float ev_ionize(const Dev& d, uint4 ci, uint64_t id, uint32_t l, PosT xn, float eps,
                                        long long born_e, long long born_i, uint3 cur,
                                        unsigned long long* qe_dst, unsigned long long* qion, BlockTally* tally)
{
    const long long ie = born_e + (long long)atomicAdd((unsigned long long*)&d.ctl->births[kE], 1ull);
    const long long ii = born_i + (long long)atomicAdd((unsigned long long*)&d.ctl->births[kI], 1ull);
    const U4x2 nb = ev_draw2(d.seed, id, l, kPurNewIon, id, l, kPurBirthId);
    const uint4 cn = nb.a, cb = nb.b;
    const uint64_t ide = child_id(cb.x, cb.y, kE), idi = child_id(cb.z, cb.w, kI);
    const U4x2 g0 = ev_draw2(d.seed, ide, l + 1, kPurGap0, idi, l + 1, kPurGap0);
    const float epr = eps - (float)kIonTh;
    const float e_ej = u23(ci.x) * epr;
    const float vs = sqrtf((epr - e_ej) * (float)(2.0 * kQE / kME));
    const float ve = sqrtf(e_ej * (float)(2.0 * kQE / kME));
    const float3 d2 = ev_iso_dir(ci.y, ci.z);
    const float2 n12 = ev_box_muller(cn.x, cn.y);
    const float2 n34 = ev_box_muller(cn.z, cn.w);
    atomicAdd(&tally->ioniz, 1u);
    const bool in_e = ie < d.cap[kE], in_i = ii < d.cap[kI];
    const SpBuf Be = d.buf[kE][cur.x];
    const SpBuf Bi = d.buf[kI][cur.y];
    if (!(in_e && in_i)) {
        atomicAdd(&tally->capacity, 1u);
        if (in_e) ((PosT*)Be.pos)[ie] = dead_value<PosT>();
        if (in_i) ((PosT*)Bi.pos)[ii] = dead_value<PosT>();
        return vs;
    }
    ((PosT*)Be.pos)[ie] = xn;
    Be.vx[ie] = ve * d2.x; Be.vy[ie] = ve * d2.y; Be.vz[ie] = ve * d2.z;
    Be.id[ie] = ide;
    Be.nev[ie] = l + ev_gap(d.lam[kE], d.lamf[kE], g0.a.x);
    ((PosT*)Bi.pos)[ii] = xn;
    Bi.vx[ii] = d.vth_gas * n12.x; Bi.vy[ii] = d.vth_gas * n12.y; Bi.vz[ii] = d.vth_gas * n34.x;
    Bi.id[ii] = idi;
    Bi.nev[ii] = l + ev_gap(d.lam[kI], d.lamf[kI], g0.b.x);
    uint32_t j, wr;
    cell_of(xn, d.kshift, j, wr);
    atomicAdd(&qe_dst[j], (1ull << 32) - wr);             // both children into this step's deposit
    if (wr) atomicAdd(&qe_dst[j + 1], (unsigned long long)wr);
    atomicAdd(&qion[j], (1ull << 32) - wr);
    if (wr) atomicAdd(&qion[j + 1], (unsigned long long)wr);
    return vs;
}

// Ar+ candidate against a gas partner w from the Maxwellian: sigma(eps) g is
// the same constant for both channels, so R nu_max < nu_cx reduces exactly
// to R < 1/2 (R on the 2^-23 grid + 1/2, never 1/2): CX gives v' = w,
// isotropic scattering v' = (v + w)/2 + |v - w|/2 n.
__device__ __noinline__ float3 ev_ion_collide(const Dev& d, uint4 c, uint64_t id, uint32_t l, float3 v,
                                              BlockTally* tally)
{
    const U4x2 g = ev_draw2(d.seed, id, l, kPurGas, id, l, kPurGas);
    const float2 n12 = ev_box_muller(g.a.x, g.a.y);
    const float2 n34 = ev_box_muller(g.a.z, g.a.w);
    const float wx = d.vth_gas * n12.x, wy = d.vth_gas * n12.y, wz = d.vth_gas * n34.x;
    if (u23(c.y) < 0.5f) {
        atomicAdd(&tally->cx, 1u);
        return make_float3(wx, wy, wz);
    }
    const float gx = v.x - wx, gy = v.y - wy, gz = v.z - wz;
    const float gm = sqrtf(gx * gx + gy * gy + gz * gz);
    const float3 dir = ev_iso_dir(c.z, c.w);
    atomicAdd(&tally->iso, 1u);
    return make_float3(0.5f * (v.x + wx) + 0.5f * gm * dir.x, 0.5f * (v.y + wy) + 0.5f * gm * dir.y,
                       0.5f * (v.z + wz) + 0.5f * gm * dir.z);
}

// Ar+ at a wall (Sec. "Wall Interaction"): energy and angle into the IEDF and
// IEADF, then sputtered-atom launch (Sec. "Wall Interactions" of the TPM):
// N = ceil(Y) trials with R <= Y/N, Thompson energy, cosine angle.
__device__ __noinline__ void ev_ion_wall(const Dev& d, uint64_t id, uint32_t l, int el, float vx, float vy, float vz,
                                         long long n_tp0, unsigned int cur_tp, BlockTally* tally)
{
    const float v2 = vx * vx + vy * vy + vz * vz;
    const float E = v2 * (float)(0.5 * kMAR / kQE);
    const float ct = fminf(v2 > 0.0f ? fabsf(vx) * rsqrtf(v2) : 1.0f, 1.0f);
    const float th = acosf(ct) * (float)(180.0 / kPI);
    hist_add(d.diag.iedf[el], kNbIedf, E, d.Emax_hist);
    const int be = hist_bin(E, d.Emax_hist, kNbIeadfE);
    const int ba = clamp_bin(th, kNbAng);
    atomicAdd(&d.diag.ieadf[el][be * kNbAng + ba], 1ull);
    atomicAdd(el == 0 ? &tally->imp_i[0] : &tally->imp_i[1], 1u);
    if (!d.sputter || !(E > (float)kSpTh)) return;
    const float Y = 0.1f * sqrtf(E / (float)kSpTh - 1.0f);
    const int Nt = min((int)ceilf(Y), kSpMaxN);
    const float Emax = lambda_ar_al() * E;
    const SpBuf T = d.buf[kTP][cur_tp];
    uint4 t = make_uint4(0, 0, 0, 0);
    for (int k = 0; k < Nt; ++k) {
        if ((k & 3) == 0) t = ev_draw2(d.seed, id, l, kPurSpTrial + (k >> 2), id, l, kPurSpTrial + (k >> 2)).a;
        const uint32_t w = (k & 3) == 0 ? t.x : (k & 3) == 1 ? t.y : (k & 3) == 2 ? t.z : t.w;
        if (!(u23(w) <= Y / (float)Nt)) continue;
        const U4x2 es = ev_draw2(d.seed, id, l, kPurSpEmit + k, id, l, kPurSpId + k);
        const float3 v = ev_emit(u23(es.a.x), u23(es.a.y), u23(es.a.z), Emax, el == 0 ? 1.0f : -1.0f);
        const long long idx = n_tp0 + (long long)atomicAdd((unsigned long long*)&d.ctl->births[kTP], 1ull);
        if (idx >= d.cap[kTP]) {
            atomicAdd(&tally->capacity, 1u);
            continue;
        }
        ((uint32_t*)T.pos)[idx] = el == 0 ? 1u : 0xffffffffu;
        T.vx[idx] = v.x;
        T.vy[idx] = v.y;
        T.vz[idx] = v.z;
        T.id[idx] = child_id(es.b.x, es.b.y, kTP);
        T.nev[idx] = 0u;
        atomicAdd(el == 0 ? &tally->sput[0] : &tally->sput[1], 1u);
    }
}

// split of the grid between the two species, proportional to their counts
// CTAs for the electrons: their share of the particles, an electron weighted
// 1.16 Ar+ (nearly all queued events are electron candidates, so an electron
// CTA's event phase is longer; at this weight the median electron and Ar+
// CTAs of the 2M + 2M sputtering discharge end together).  Results do not
// depend on the division.
constexpr float kElectronWeight = 1.16f;
__device__ __forceinline__ int electron_ctas(long long ne, long long ni, int G)
{
    if (ne <= 0) return 0;
    if (ni <= 0) return G;
    const float we = kElectronWeight * (float)ne;
    int Ge = (int)((float)G * (we / (we + (float)ni)) + 0.5f);
    return Ge < 1 ? 1 : (Ge > G - 1 ? G - 1 : Ge);
}

__device__ __forceinline__ void flush_tally(const Dev& d, const BlockTally& t, int cta)
{
    unsigned long long* r = d.tally + (size_t)cta * kNumCnt;
    const unsigned int v[13] = {t.elastic, t.excit, t.ioniz, t.cx, t.iso, t.imp_e[0], t.imp_e[1],
                                t.numerics, t.capacity, t.imp_i[0], t.imp_i[1], t.sput[0], t.sput[1]};
    const int k[13] = {kCntElastic, kCntExcit, kCntIoniz, kCntCx, kCntIso, kCntImpEL, kCntImpER,
                       kCntNumerics, kCntCapacity, kCntImpIL, kCntImpIR, kCntSputL, kCntSputR};
#pragma unroll
    for (int i = 0; i < 13; ++i)
        if (v[i]) atomicAdd(&r[k[i]], (unsigned long long)v[i]);
    if (t.numerics) atomicOr(&d.ctl->err, kErrNumerics);
    if (t.capacity) atomicOr(&d.ctl->err, kErrCapacity);
    if (d.circuit) {                              // charge delivered to the driven electrode
        const long long dn = (long long)t.imp_i[0] - (long long)t.imp_e[0];
        if (dn) atomicAdd((unsigned long long*)&d.ctl->wall_delta, (unsigned long long)dn);
    }
}

// ---------------------------------------------------------------- mover
// Slots are streamed in groups of four (16-byte vector loads and stores);
// consecutive threads take consecutive groups.  A step reads x, v_x and the
// step of the next null-collision candidate and writes x and v_x; v_y, v_z
// and the id are touched only by events.  Electrons reaching a wall are
// counted in registers; Ar+ wall hits and collision candidates (well under
// 1% of the particles per step) are queued in shared memory and handled after
// the streaming loop; births go to slots from round_up(n, 4) on, which no
// vector store of this launch touches.
constexpr int kQueueCap = 1024;
enum : uint32_t { kEvCand = 0u, kEvWallL = 1u, kEvWallR = 2u };

template <bool P64> struct Pos4;
template <> struct Pos4<false> {
    uint4 v;
    __device__ __forceinline__ void load(const void* base, long long g) { v = ((const uint4*)base)[g]; }
    __device__ __forceinline__ void store(void* base, long long g) const { ((uint4*)base)[g] = v; }
    __device__ __forceinline__ uint32_t get(int u) const { return u == 0 ? v.x : u == 1 ? v.y : u == 2 ? v.z : v.w; }
    __device__ __forceinline__ void set(int u, uint32_t x)
    {
        if (u == 0) v.x = x; else if (u == 1) v.y = x; else if (u == 2) v.z = x; else v.w = x;
    }
};
template <> struct Pos4<true> {
    double2 a, b;
    __device__ __forceinline__ void load(const void* base, long long g)
    {
        a = ((const double2*)base)[2 * g];
        b = ((const double2*)base)[2 * g + 1];
    }
    __device__ __forceinline__ void store(void* base, long long g) const
    {
        ((double2*)base)[2 * g] = a;
        ((double2*)base)[2 * g + 1] = b;
    }
    __device__ __forceinline__ double get(int u) const { return u == 0 ? a.x : u == 1 ? a.y : u == 2 ? b.x : b.y; }
    __device__ __forceinline__ void set(int u, double x)
    {
        if (u == 0) a.x = x; else if (u == 1) a.y = x; else if (u == 2) b.x = x; else b.y = x;
    }
};

__device__ __forceinline__ float f4get(const float4& v, int u) { return u == 0 ? v.x : u == 1 ? v.y : u == 2 ? v.z : v.w; }
__device__ __forceinline__ void f4set(float4& v, int u, float x)
{
    if (u == 0) v.x = x; else if (u == 1) v.y = x; else if (u == 2) v.z = x; else v.w = x;
}

__device__ __forceinline__ long long round4(long long n) { return (n + 3) & ~3ll; }


// Shared-memory accumulators of one CTA.  The linear weights are summed per
// cell in three 32-bit counters -- particles n_j, and the high and low 16 bits
// of their right-node weights wr -- so that node m receives
//     n_m 2^32 - (hi_m 2^16 + lo_m) + (hi_{m-1} 2^16 + lo_{m-1}),
// exactly as the per-particle rule would give.  32-bit shared atomics are
// native; with at most 65536 particles per tile no counter can overflow.
// The flux moment uses 64-bit sums kept as (low, high) 32-bit pairs with the
// carry propagated from the low word's atomic return value.
constexpr long long kTileGroups = 16384;     // 65536 particles

// bytes of the region shared by the field-solve copies (2 x u64 [N+1]) and
// the tile sums (3 x u32 [N] + 2 x u32 [N+1]), rounded to 16
__host__ __device__ __forceinline__ size_t q_bytes16(int N) { return ((size_t)(N + 1) * 8 + 15) & ~(size_t)15; }
__host__ __device__ __forceinline__ size_t acc_bytes(int N)
{
    return ((size_t)N * 12 + (size_t)(N + 1) * 8 + 15) & ~(size_t)15;
}

struct Acc {
    unsigned int* cnt;   // [N]
    unsigned int* whi;   // [N]
    unsigned int* wlo;   // [N]
    unsigned int* flo;   // [N+1]
    int* fhi;            // [N+1]
};

__device__ __forceinline__ void acc_add64(unsigned int* lo, int* hi, int m, long long v)
{
    const unsigned int vl = (unsigned int)v;
    const unsigned int old = atomicAdd(&lo[m], vl);
    const int carry = old + vl < old ? 1 : 0;
    const int vh = (int)(v >> 32) + carry;
    if (vh) atomicAdd(&hi[m], vh);
}

// Deposit of one group of four slots into the tile sums.  When every active
// lane of the warp holds four particles of one and the same cell (cell-sorted,
// slow particles), the warp sums its weights with REDUX and one lane adds
// them; otherwise one set of atomics per group when its four slots share a
// cell, else one set per particle.  On sample steps also the flux moment.
__device__ __forceinline__ void deposit_group(const Acc& A, const bool (&dep)[4], const uint32_t (&j)[4],
                                              const uint32_t (&wr)[4], const float (&vx)[4], bool sample)
{
    const bool one = dep[0] && dep[1] && dep[2] && dep[3] && j[0] == j[1] && j[1] == j[2] && j[2] == j[3];
    const uint32_t h = (wr[0] >> 16) + (wr[1] >> 16) + (wr[2] >> 16) + (wr[3] >> 16);
    const uint32_t lo = (wr[0] & 0xffffu) + (wr[1] & 0xffffu) + (wr[2] & 0xffffu) + (wr[3] & 0xffffu);
    const unsigned m = __activemask();
    const int leader = __ffs(m) - 1;
    const uint32_t jl = __shfl_sync(m, j[0], leader);
    if (__all_sync(m, one && j[0] == jl)) {
        const uint32_t hs = __reduce_add_sync(m, h), ls = __reduce_add_sync(m, lo);
        if ((int)(threadIdx.x & 31) == leader) {
            atomicAdd(&A.cnt[jl], 4u * (unsigned)__popc(m));
            atomicAdd(&A.whi[jl], hs);
            atomicAdd(&A.wlo[jl], ls);
        }
    } else if (one) {
        atomicAdd(&A.cnt[j[0]], 4u);
        atomicAdd(&A.whi[j[0]], h);
        atomicAdd(&A.wlo[j[0]], lo);
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (!dep[u]) continue;
            atomicAdd(&A.cnt[j[u]], 1u);
            atomicAdd(&A.whi[j[u]], wr[u] >> 16);
            atomicAdd(&A.wlo[j[u]], wr[u] & 0xffffu);
        }
    }
    if (sample) {
        if (one) {                            // four particles of one cell: one pair of sums
            long long f0 = 0, f1 = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long vq = (long long)__float2int_rn(vx[u]);
                const long long w16 = (long long)(wr[u] >> 16);
                f0 += vq * (65536 - w16);
                f1 += vq * w16;
            }
            acc_add64(A.flo, A.fhi, j[0], f0);
            acc_add64(A.flo, A.fhi, j[0] + 1, f1);
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (!dep[u]) continue;
                const long long vq = (long long)__float2int_rn(vx[u]);
                const long long w16 = (long long)(wr[u] >> 16);
                acc_add64(A.flo, A.fhi, j[u], vq * (65536 - w16));
                acc_add64(A.flo, A.fhi, j[u] + 1, vq * w16);
            }
        }
    }
}

// One queued event: a collision candidate of either species (Sec. "Particle
// Collisions"), or an Ar+ wall hit.  e- candidates: the process by R nu_max
// against the cumulative nu_el, nu_exc, nu_ion at the electron's energy;
// isotropic scattering; elastic loss 2 m_e/M (1 - cos chi); excitation
// -11.5 eV; ionisation in ev_ionize.  Every candidate draws the step of its
// next candidate.
template <typename PosT>
__device__ __noinline__ void handle_event(const Dev& d, int s, long long i, uint32_t kind, uint32_t l,
                                          long long born_e, long long born_i, long long ntp, uint3 cur,
                                          unsigned long long* qe_dst, unsigned long long* qion,
                                          BlockTally* tally)
{
    const SpBuf B = d.buf[s][s == kE ? cur.x : cur.y];
    float vx = B.vx[i], vy = B.vy[i], vz = B.vz[i];
    const uint64_t id = B.id[i];
    if (kind != kEvCand) {
        const int el = kind == kEvWallL ? 0 : 1;
        if (s == kI) ev_ion_wall(d, id, l, el, vx, vy, vz, ntp, cur.z, tally);
        else atomicAdd(&tally->imp_e[el], 1u);          // (electrons at a wall are counted in the stream)
        return;
    }
    const U4x2 cg = ev_draw2(d.seed, id, l, kPurColl, id, l, kPurGap);
    const uint4 c = cg.a;
    B.nev[i] = l + ev_gap(d.lam[s], d.lamf[s], cg.b.x);
    if (s == kE) {
        const float v2 = vx * vx + vy * vy + vz * vz;
        const float v = sqrtf(v2);
        const float eps = v2 * (float)(0.5 * kME / kQE);
        if (eps > d.eps_max) atomicAdd(&tally->numerics, 1u);
        float s_el = (float)kSigEl;
        float s_exc = eps > (float)kExcTh ? (float)kExcSig * (1.0f - (float)kExcTh / eps) : 0.0f;
        float s_ion = eps > (float)kIonTh
                          ? (float)(kLotzA * kLotzQ) * logf(eps / (float)kIonTh) / (eps * (float)kIonTh)
                          : 0.0f;
        if (d.xs_n[0] | d.xs_n[1] | d.xs_n[2]) {
            if (d.xs_n[0]) s_el = ev_xs_table(d.xs_tab[0], d.xs_n[0], eps);
            if (d.xs_n[1]) s_exc = ev_xs_table(d.xs_tab[1], d.xs_n[1], eps);
            if (d.xs_n[2]) s_ion = ev_xs_table(d.xs_tab[2], d.xs_n[2], eps);
        }
        const float nu_el = d.ngas_f * s_el * v;
        const float nu_exc = d.ngas_f * s_exc * v;
        const float nu_ion = d.ngas_f * s_ion * v;
        const float r = u23(c.y) * d.nu_max_e;
        const float3 dir = iso_dir(c.z, c.w);
        float vn = -1.0f;
        if (r < nu_el) {
            const float cchi = v > 0.0f ? (dir.x * vx + dir.y * vy + dir.z * vz) / v : 1.0f;
            vn = v * sqrtf(1.0f - (float)(2.0 * kME / kMAR) * (1.0f - cchi));
            atomicAdd(&tally->elastic, 1u);
        } else if (r < nu_el + nu_exc) {
            vn = sqrtf((eps - (float)kExcTh) * (float)(2.0 * kQE / kME));
            atomicAdd(&tally->excit, 1u);
        } else if (r < nu_el + nu_exc + nu_ion) {
            const uint4 ci = ev_draw2(d.seed, id, l, kPurIonize, id, l, kPurIonize).a;
            vn = ev_ionize<PosT>(d, ci, id, l, ((const PosT*)B.pos)[i], eps, born_e, born_i, cur, qe_dst, qion,
                                 tally);
        }
        if (vn >= 0.0f) {
            vx = vn * dir.x; vy = vn * dir.y; vz = vn * dir.z;
        }
    } else {
        const float3 nv = ev_ion_collide(d, c, id, l, make_float3(vx, vy, vz), tally);
        vx = nv.x; vy = nv.y; vz = nv.z;
    }
    B.vx[i] = vx;
    B.vy[i] = vy;
    B.vz[i] = vz;
}

template <bool P64>
struct Grp {                   // one group of four slots, as loaded
    Pos4<P64> p;
    float4 v;
    uint4 nv;                  // steps of the next candidate
    float4 vy, vz;             // electrons on sample steps (EEDF)
};

template <bool P64, int MODE, bool SAMPLE>
__device__ __forceinline__ Grp<P64> load_group(const SpBuf& B, long long g, bool eedf)
{
    Grp<P64> G;
    G.p.load(B.pos, g);
    if (MODE == 0) {
        G.v = ((const float4*)B.vx)[g];
        G.nv = ((const uint4*)B.nev)[g];
        if (SAMPLE && eedf) {
            G.vy = ((const float4*)B.vy)[g];
            G.vz = ((const float4*)B.vz)[g];
        }
    }
    return G;
}

// node totals of the tile into the global histograms; clear the tile sums
// when another tile follows
__device__ void flush_tile(const Acc& A, int N, unsigned int jlo, unsigned int jhi, bool sample,
                           unsigned long long* qdst, long long* fdst, bool clear, int t, int nt)
{
    if (jlo != 0xffffffffu) {
        for (int m = (int)jlo + t; m <= (int)jhi + 1; m += nt) {
            unsigned long long v = 0;
            if (m < N) v += ((unsigned long long)A.cnt[m] << 32) - (((unsigned long long)A.whi[m] << 16) + A.wlo[m]);
            if (m > 0) v += ((unsigned long long)A.whi[m - 1] << 16) + A.wlo[m - 1];
            if (v) atomicAdd(&qdst[m], v);
            if (sample) {
                const long long f = (long long)(((unsigned long long)(unsigned int)A.fhi[m] << 32) | A.flo[m]);
                if (f) atomicAdd((unsigned long long*)&fdst[m], (unsigned long long)f);
            }
        }
    }
    if (!clear) return;
    __syncthreads();
    for (int m = t; m <= N; m += nt) {
        if (m < N) A.cnt[m] = A.whi[m] = A.wlo[m] = 0;
        A.flo[m] = 0;
        A.fhi[m] = 0;
    }
}

// MODE 0: full PIC/MCC step.  MODE 1: deposit the current state (creation,
// after a state upload).  Slots are streamed in groups of four with 16-byte
// vector loads and stores; consecutive threads take consecutive groups and
// each thread loads its next group before working on the current one.
// The body of one step launch for one discharge, run by CTA `cta` of the
// `ncta` CTAs the discharge has in the launch.
// reuse_field: the CTA ran the previous body call for the same discharge and
// step, so its shared memory already holds that step's deposit and field.
template <bool P64, int MODE, bool SAMPLE>
__device__ __forceinline__ void mover_body(const Dev& d, const StepArgs& a, int cta, int ncta, bool sample_on = true,
                                           bool reuse_field = false)
{
    using PosT = typename std::conditional<P64, double, uint32_t>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = d.ncell, N1 = N + 1;
    // layout: [qe u64 N1 | qi u64 N1, each padded to 16 bytes] [tile sums] [sEd float2 N]
    //         [sE float N1] [eedf u32 256] [queue u32 kQueueCap]
    unsigned long long* sqe = (unsigned long long*)smem_raw;
    unsigned long long* sqi = (unsigned long long*)(smem_raw + q_bytes16(N));
    unsigned char* sacc = smem_raw + 2 * q_bytes16(N);
    Acc A;
    A.cnt = (unsigned int*)sacc;
    A.whi = A.cnt + N;
    A.wlo = A.whi + N;
    A.flo = A.wlo + N;
    A.fhi = (int*)(A.flo + N1);
    float2* sEd = (float2*)(sacc + acc_bytes(N));
    float* sE = (float*)(sEd + N);
    unsigned int* seedf = (unsigned int*)(sE + N1);
    unsigned int* squeue = seedf + kNbEedf;
    __shared__ BlockTally tally;
    __shared__ unsigned int s_jlo, s_jhi, s_qn;
    __shared__ int s_last, s_overflow;
    __shared__ unsigned long long s_evmax, s_flushns;
    __shared__ double s_vel;                    // electrode potential of the field in shared memory

    unsigned long long* tr = d.trace ? d.trace + (size_t)cta * kTraceSlots : nullptr;
    if (tr && threadIdx.x == 0) tr[0] = gtimer();
    const unsigned int l = a.step;              // the host's step count (equal to ctl->step)
    Ctl* ctl = d.ctl;
    const long long ne = ctl->n[kE], ni = ctl->n[kI], ntp = ctl->n[kTP];
    // charge delivered to the driven electrode (series capacitor), loaded now so
    // that its latency passes during the deposit copy
    const long long wall_dn = MODE == 0 && a.field_mode == kFieldCircuit ? ctl->wall_dn : 0ll;
    const unsigned int field_override = MODE == 0 ? ctl->field_override : 0u;
    if (MODE == 0 && !reuse_field) {
        // both deposits of x^l (slot l%3) into shared memory: asynchronous
        // 16-byte copies, all in flight at once (arrays 256-byte aligned, padded)
        const int slot = l % 3;
        const int nv = (N1 * 8 + 15) / 16;
        for (int i = threadIdx.x; i < 2 * nv; i += blockDim.x) {
            const int sp = i < nv ? kE : kI, k = i < nv ? i : i - nv;
            const char* src = (const char*)d.qbuf[slot][sp] + 16 * k;
            char* dst = (char*)(sp == kE ? sqe : sqi) + 16 * k;
            const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src) : "memory");
        }
    }
    // sample steps (flux moment, EEDF) are a separate instantiation: the host
    // launches it when (l + 1) % diag_every == 0
    const bool sample = MODE == 0 && SAMPLE && sample_on;
    const int G = ncta;
    const int Ge = electron_ctas(ne, ni, G);
    const int s = (int)cta < Ge ? kE : kI;
    const int b = s == kE ? cta : cta - Ge;
    const int Gs = s == kE ? Ge : G - Ge;
    const long long ns = s == kE ? ne : ni;
    const long long G4 = (ns + 3) >> 2;
    const long long per = G4 / Gs, extra = G4 - per * Gs;     // balanced split of the groups
    const long long cg0 = (long long)b * per + min((long long)b, extra);
    const long long cg1 = cg0 + per + (b < extra ? 1 : 0);
    const long long T = blockDim.x;
    const long long chunk0 = 4 * cg0;
    const int dslot = MODE == 0 ? (l + 1) % 3 : l % 3;
    unsigned long long* qdst = d.qbuf[dslot][s];
    unsigned long long* qe_dst = d.qbuf[dslot][kE];
    unsigned long long* qion = d.qbuf[dslot][kI];
    long long* fdst = d.fbuf[dslot][s];
    const SpBuf B = d.buf[s][a.cur[s]];
    if (tr && threadIdx.x == 0) tr[10] = gtimer();

    // first group of this thread: in flight during the field solve
    long long g = cg0 + threadIdx.x;
    const long long tile1_first = min(cg1, cg0 + kTileGroups);
    Grp<P64> nxt;
    if (g < tile1_first) nxt = load_group<P64, MODE, SAMPLE>(B, g, s == kE && sample);
    if (tr && threadIdx.x == 0) tr[11] = gtimer();

    {
        // work that needs no deposit, while its copies are in flight: clear the
        // tile sums (cnt, whi, wlo, flo, fhi are contiguous) and the EEDF tally,
        // and this CTA's share of slot (l+2)%3 (read by the previous launch,
        // deposited into by the next)
        const int t = threadIdx.x, nt = blockDim.x;
        uint4* z4 = (uint4*)A.cnt;
        for (int k = t; k < (int)(acc_bytes(N) / 16); k += nt) z4[k] = make_uint4(0u, 0u, 0u, 0u);
        for (int i = t; i < kNbEedf; i += nt) seedf[i] = 0;
        if (t == 0) {
            tally = BlockTally{};
            s_jlo = 0xffffffffu;
            s_jhi = 0;
            s_qn = 0;
            s_overflow = 0;
            s_evmax = 0;
            s_flushns = 0;
        }
        if (MODE == 0) {
            const int m0 = N1 * cta / G, m1 = N1 * (cta + 1) / G;
            const int z = (l + 2) % 3;
            for (int i = m0 + t; i < m1; i += nt) {
                d.qbuf[z][kE][i] = 0;
                d.qbuf[z][kI][i] = 0;
                d.fbuf[z][kE][i] = 0;
                d.fbuf[z][kI][i] = 0;
            }
        }
    }
    if (MODE == 0) asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    if (tr && threadIdx.x == 0) tr[1] = gtimer();
    double v_el = a.v_left;                     // electrode potential of step l
    if (MODE == 0 && !reuse_field) {
        // field of step l: every CTA solves from the deposit of x^l
        if (field_override) {
            for (int i = threadIdx.x; i < N1; i += blockDim.x) sE[i] = d.E32[i];
        } else {
            v_el = block_field_f32(d, sqe, sqi, sE, a, wall_dn);
        }
        if (threadIdx.x == 0) s_vel = v_el;
    }
    __syncthreads();
    if (tr && threadIdx.x == 0) tr[2] = gtimer();
    if (MODE == 0 && !reuse_field) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) sEd[i] = make_float2(sE[i], sE[i + 1] - sE[i]);
        __syncthreads();
    }
    if (reuse_field) v_el = s_vel;
    if (tr && threadIdx.x == 0) tr[3] = gtimer();

    const float qmdt = d.qm_dt[s];
    const long long born_e = round4(ne), born_i = round4(ni);
    const uint3 cur3 = make_uint3(a.cur[kE], a.cur[kI], a.cur[kTP]);
    const PosT dead = dead_value<PosT>();
    uint32_t jlo = 0xffffffffu, jhi = 0;
    unsigned int imp_l = 0, imp_r = 0;          // electrons absorbed at x = 0 / x = L

    for (long long t0 = cg0; t0 < cg1; t0 += kTileGroups) {
        const long long t1 = min(cg1, t0 + kTileGroups);
        if (t0 > cg0) {                               // next tile: flush the sums of the last one
            const unsigned int lo = __reduce_min_sync(0xffffffffu, jlo), hi = __reduce_max_sync(0xffffffffu, jhi);
            if ((threadIdx.x & 31) == 0) {
                atomicMin(&s_jlo, lo);
                atomicMax(&s_jhi, hi);
            }
            __syncthreads();
            flush_tile(A, N, s_jlo, s_jhi, sample, qdst, fdst, true, threadIdx.x, blockDim.x);
            __syncthreads();
            if (threadIdx.x == 0) {
                s_jlo = 0xffffffffu;
                s_jhi = 0;
            }
            jlo = 0xffffffffu;
            jhi = 0;
            g = t0 + threadIdx.x;
            if (g < t1) nxt = load_group<P64, MODE, SAMPLE>(B, g, s == kE && sample);
            __syncthreads();
        }
        while (g < t1) {
            Grp<P64> Gc = nxt;
            const long long gn = g + T;
            if (gn < t1) nxt = load_group<P64, MODE, SAMPLE>(B, gn, s == kE && sample);
            if (4 * g + 4 > ns) {                     // the species' last group: slots past n are removed
                const int rem = (int)(ns - 4 * g);
#pragma unroll
                for (int u = 1; u < 4; ++u)
                    if (u >= rem) Gc.p.set(u, dead);
            }
            PosT x[4];
            bool act[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                x[u] = Gc.p.get(u);
                act[u] = is_alive(x[u]);
                if (P64 && act[u] && !((double)x[u] < (double)N)) {
                    act[u] = false;
                    atomicOr(&ctl->err, kErrIndex);
                }
            }
            uint32_t j[4], wr[4];
            bool dep[4];
            float vx[4] = {Gc.v.x, Gc.v.y, Gc.v.z, Gc.v.w};
            if (MODE == 1) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    dep[u] = act[u];
                    cell_of(act[u] ? x[u] : (PosT)(P64 ? 0.5 : 1.0), d.kshift, j[u], wr[u]);
                    if (dep[u]) {
                        jlo = min(jlo, j[u]);
                        jhi = max(jhi, j[u]);
                    }
                }
                deposit_group(A, dep, j, wr, vx, false);
                Gc.p.store(B.pos, g);
                g = gn;
                continue;
            }
            // gather + leapfrog for the four slots (branch-free; removed slots are ignored later)
            PosT xn[4];
            uint32_t kind[4];
            const uint32_t nv[4] = {Gc.nv.x, Gc.nv.y, Gc.nv.z, Gc.nv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                uint32_t jj, ww;                       // (32-bit: a removed slot, 0, reads cell 0)
                cell_of(P64 && !act[u] ? (PosT)0.5 : x[u], d.kshift, jj, ww);
                const float2 e = sEd[jj];
                const float f = __uint_as_float(0x3f800000u | (ww >> 9)) - 1.0f;
                vx[u] = vx[u] + qmdt * (e.x + f * e.y);
                if (P64) {
                    const double xd = (double)x[u] + (double)vx[u] * d.push64;
                    kind[u] = xd <= 0.0 ? kEvWallL : (xd >= (double)N ? kEvWallR : 0xffffffffu);
                    xn[u] = (PosT)xd;
                } else {
                    const int disp = __float2int_rn(vx[u] * d.push32);
                    const uint32_t xu = (uint32_t)x[u];
                    const uint32_t xm = xu + (uint32_t)disp;
                    kind[u] = (disp > 0 && xm < xu) ? kEvWallR
                              : ((disp < 0 && (0u - (uint32_t)disp) >= xu) ? kEvWallL : 0xffffffffu);
                    xn[u] = (PosT)xm;
                }
            }
            uint32_t evm = 0;                          // bit u: slot u goes to the event queue
            uint32_t wlm = 0, wrm = 0;                 // bit u: slot u left at x = 0 / x = L
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                dep[u] = act[u] && kind[u] == 0xffffffffu;
                // (32-bit: a position that left the gap wrapped around and still names a cell)
                cell_of(P64 && !dep[u] ? (PosT)0.5 : xn[u], d.kshift, j[u], wr[u]);
                Gc.p.set(u, dep[u] ? xn[u] : dead);
                jlo = min(jlo, dep[u] ? j[u] : 0xffffffffu);
                jhi = max(jhi, dep[u] ? j[u] : 0u);
                const bool wall = act[u] && !dep[u];
                const bool cand = dep[u] && (int)(nv[u] - l) <= 0;
                if (cand) kind[u] = kEvCand;
                wlm |= (wall && kind[u] == kEvWallL) ? 1u << u : 0u;
                wrm |= (wall && kind[u] == kEvWallR) ? 1u << u : 0u;
                evm |= cand ? 1u << u : 0u;
            }
            if (s == kE) {                             // an electron at a wall is only counted
                if (wlm | wrm) {
                    imp_l += __popc(wlm);
                    imp_r += __popc(wrm);
                }
            } else {
                evm |= wlm | wrm;
            }
            deposit_group(A, dep, j, wr, vx, sample);
            if (sample && s == kE) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (!dep[u]) continue;
                    bool inwin;
                    if (P64) inwin = (double)xn[u] >= d.eedf_lo64 && (double)xn[u] < d.eedf_hi64;
                    else inwin = (uint32_t)xn[u] >= d.eedf_lo && (uint32_t)xn[u] < d.eedf_hi;
                    if (inwin) {
                        const float vy = f4get(Gc.vy, u), vz = f4get(Gc.vz, u);
                        const float en = (vx[u] * vx[u] + vy * vy + vz * vz) * (float)(0.5 * kME / kQE);
                        atomicAdd(&seedf[hist_bin(en, 64.0f, kNbEedf)], 1u);
                    }
                }
            }
            if (evm) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (!(evm & (1u << u))) continue;
                    const long long i = 4 * g + u;
                    // the event reads v_y, v_z and the id, which the stream does not
                    // load: bring their lines to L2 now, well before it runs
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(B.vy + i));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(B.vz + i));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(B.id + i));
                    const unsigned int q = atomicAdd(&s_qn, 1u);
                    if (q < (unsigned)kQueueCap) {
                        squeue[q] = ((uint32_t)(i - chunk0) << 2) | kind[u];
                    } else {                            // queue full: flag the slot
                        d.evflag[s][i] = (unsigned char)(kind[u] + 1u);
                        s_overflow = 1;
                    }
                }
            }
            Gc.p.store(B.pos, g);
            ((float4*)B.vx)[g] = make_float4(vx[0], vx[1], vx[2], vx[3]);
            g = gn;
        }
    }
    if (MODE == 0 && s == kE) {
        imp_l = __reduce_add_sync(0xffffffffu, imp_l);
        imp_r = __reduce_add_sync(0xffffffffu, imp_r);
        if ((threadIdx.x & 31) == 0 && (imp_l | imp_r)) {
            atomicAdd(&tally.imp_e[0], imp_l);
            atomicAdd(&tally.imp_e[1], imp_r);
        }
    }
    // range of touched nodes
    jlo = __reduce_min_sync(0xffffffffu, jlo);
    jhi = __reduce_max_sync(0xffffffffu, jhi);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&s_jlo, jlo);
        atomicMax(&s_jhi, jhi);
    }
    __syncthreads();
    if (tr && threadIdx.x == 0) tr[4] = gtimer();
    // queued events on the first half of the CTA, node totals of the tile on
    // the second half (the events deposit their births globally)
    const int half = blockDim.x / 2;
    if (MODE == 0 && (int)threadIdx.x < half) {
        const unsigned int qn = min(s_qn, (unsigned)kQueueCap);
        for (unsigned int k = threadIdx.x; k < qn; k += half) {
            const uint32_t e = squeue[k];
            const unsigned long long te = tr ? gtimer() : 0ull;
            handle_event<PosT>(d, s, chunk0 + (e >> 2), e & 3u, l, born_e, born_i, ntp, cur3, qe_dst, qion,
                               &tally);
            if (tr) atomicMax(&s_evmax, ((gtimer() - te) << 8) | (e & 3u));
        }
    } else {
        const int t = MODE == 0 ? threadIdx.x - half : threadIdx.x;
        const int nt = MODE == 0 ? blockDim.x - half : blockDim.x;
        const unsigned long long tf = tr ? gtimer() : 0ull;
        flush_tile(A, N, s_jlo, s_jhi, sample, qdst, fdst, false, t, nt);
        if (tr) atomicMax(&s_flushns, gtimer() - tf);
        if (MODE == 0 && a.accumulate) {         // this CTA's share of the time averages of step l
            const int m0 = N1 * cta / G, m1 = N1 * (cta + 1) / G;
            accumulate_nodes(d, l, sqe, sqi, m0, m1, v_el, cta == 0, t, nt);
        }
    }
    if (MODE == 0 && s_overflow) {
        const long long chunk1 = min(4 * cg1, ns);
        for (long long i = chunk0 + threadIdx.x; i < chunk1; i += blockDim.x) {
            const unsigned char k = d.evflag[s][i];
            if (k) {
                d.evflag[s][i] = 0;
                handle_event<PosT>(d, s, i, k - 1u, l, born_e, born_i, ntp, cur3, qe_dst, qion, &tally);
            }
        }
    }
    if (tr && threadIdx.x == 0) {
        tr[5] = gtimer();
        tr[8] = (unsigned long long)s;
        tr[9] = (unsigned long long)s_qn | ((unsigned long long)(s_jhi - s_jlo + 1u) << 32);
    }
    __syncthreads();
    if (sample && s == kE)
        for (int i = threadIdx.x; i < kNbEedf; i += blockDim.x)
            if (seedf[i]) atomicAdd(&d.diag.eedf[i], (unsigned long long)seedf[i]);
    if (threadIdx.x == 0) flush_tally(d, tally, cta);
    if (tr && threadIdx.x == 0) {
        tr[6] = gtimer();
        tr[12] = s_evmax;
        tr[13] = tally.ioniz;
        tr[14] = s_flushns;
    }
    // last CTA: commit the step
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ctl->done, 1u) == (unsigned)(G - 1);
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        commit_step(d, MODE == 0);
    }
    if (tr && threadIdx.x == 0) tr[7] = gtimer();
}

template <bool P64, int MODE, bool SAMPLE>
__global__ void __launch_bounds__(kMoverThreads, kMoverMinBlocks) k_mover(Dev d, StepArgs a)
{
    // Launched with programmatic stream serialization: the next launch in the
    // stream may place its CTAs on SMs as this launch's CTAs exit, and every
    // CTA waits here until the previous launch has completed and its writes
    // are visible (a hardware dependency, not a spin), before any global access.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    mover_body<P64, MODE, SAMPLE>(d, a, blockIdx.x, gridDim.x);
}

// One PIC/MCC step of every discharge of a batch in one launch.  Each CTA
// belongs to one discharge (owner[]), copies that discharge's descriptor and
// step arguments into shared memory and runs the step kernel's body for it;
// the discharges' results do not depend on which others share the launch.
template <bool SAMPLE>
__global__ void __launch_bounds__(kMoverThreads, kMoverMinBlocks)
    k_mover_batch(const BatchEntry* __restrict__ ent, const int* __restrict__ owner)
{
    __shared__ __align__(16) Dev sd;
    __shared__ StepArgs sa;
    __shared__ int s_k;
    if (threadIdx.x == 0) s_k = owner[blockIdx.x];
    __syncthreads();
    const BatchEntry& e = ent[s_k];
    const unsigned int* src = (const unsigned int*)&e.d;
    unsigned int* dst = (unsigned int*)&sd;
    for (int i = threadIdx.x; i < (int)(sizeof(Dev) / 4); i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x == 0) {
        const Ctl* c = e.d.ctl;
        const unsigned int l = c->step;
        StepArgs a = e.phase[l % e.period];
        a.step = l;
        a.accumulate = l >= e.acc_from ? 1 : 0;
        a.cur[0] = c->cur[0];
        a.cur[1] = c->cur[1];
        a.cur[2] = c->cur[2];
        sa = a;
    }
    __syncthreads();
    mover_body<false, 0, SAMPLE>(sd, sa, (int)blockIdx.x - e.cta0, e.ncta);
}

// The batched step with resident CTAs: the launch has a few CTAs per SM, and
// each takes chunks of consecutive CTA slots of one discharge from a work
// counter (chunks[c]: discharge, first and last slot).  A chunk's slots run
// one after another through the step body; the first pays the deposit copy
// and field solve of that discharge, the others reuse them.  work[0] hands
// out chunks, work[1] counts the CTAs that have finished; the last resets both
// for the next launch.
template <bool SAMPLE>
__global__ void __launch_bounds__(kMoverThreads, kMoverMinBlocks)
    k_mover_batch_chunks(const BatchEntry* __restrict__ ent, const BatchChunk* __restrict__ chunks, int nchunks,
                         unsigned int* work)
{
    __shared__ __align__(16) Dev sd;
    __shared__ StepArgs sa;
    __shared__ int s_c, s_member;
    if (threadIdx.x == 0) s_member = -1;
    for (;;) {
        __syncthreads();                          // the previous body (and its commit) are done
        if (threadIdx.x == 0) s_c = (int)atomicAdd(&work[0], 1u);
        __syncthreads();
        const int c = s_c;
        if (c >= nchunks) break;
        const BatchChunk ch = chunks[c];
        const bool same = ch.member == s_member;
        if (!same) {
            const BatchEntry& e = ent[ch.member];
            const unsigned int* src = (const unsigned int*)&e.d;
            unsigned int* dst = (unsigned int*)&sd;
            for (int i = threadIdx.x; i < (int)(sizeof(Dev) / 4); i += blockDim.x) dst[i] = src[i];
            if (threadIdx.x == 0) {
                const Ctl* cc = e.d.ctl;
                const unsigned int l = cc->step;
                StepArgs a = e.phase[l % e.period];
                a.step = l;
                a.accumulate = l >= e.acc_from ? 1 : 0;
                a.cur[0] = cc->cur[0];
                a.cur[1] = cc->cur[1];
                a.cur[2] = cc->cur[2];
                sa = a;
                s_member = ch.member;
            }
            __syncthreads();
        }
        const int ncta = ent[ch.member].ncta;
        for (int v = ch.v0; v < ch.v1; ++v) {
            mover_body<false, 0, SAMPLE>(sd, sa, v, ncta, true, same || v > ch.v0);
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&work[1], 1u) == gridDim.x - 1) {
            work[0] = 0;
            work[1] = 0;
            __threadfence();
        }
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

// FP64 field and potential of the current state (step l, slot l%3), for
// diagnostics; optionally adds step l to the time averages if no launch has.
__global__ void k_field(Dev d, double v_left, int accumulate)
{
    const unsigned int l = d.ctl->step;
    const int slot = l % 3;
    QNet qn{d.qbuf[slot][kI], d.qbuf[slot][kE], false};
    const CircuitArgs circ{d.circ_a, d.circ_b, d.ctl->wall_dn};
    const double v_el = poisson_block(qn, d.ncell, d.A, d.inv_dx, v_left, d.phi, d.E64, nullptr,
                                      d.circuit && d.A > 0.0 ? &circ : nullptr);
    __syncthreads();
    if (accumulate)
        accumulate_nodes(d, l, d.qbuf[slot][kE], d.qbuf[slot][kI], 0, d.ncell + 1, v_el, true, threadIdx.x,
                         blockDim.x);
}

// ---------------------------------------------------------------- uploaded state
__global__ void k_entry_nev(Dev d, int s, unsigned int half, long long n, unsigned int l0)
{
    const SpBuf B = d.buf[s][half];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        B.nev[k] = entry_nev(d, s, B.id[k], l0);
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
    // a contiguous run of slots per CTA: cell-ordered runs touch few cells, so
    // few global atomics follow
    const long long i0 = n * blockIdx.x / gridDim.x, i1 = n * (blockIdx.x + 1) / gridDim.x;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
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

// Scatter straight from registers (the Ar+, which stay cell-ordered between
// compactions, so a warp's particles fall in one or two cells and its stores
// are already runs): each CTA takes a contiguous run of slots, counts its
// particles per cell in shared memory, reserves one sub-range per touched
// cell of the cell's global range (one global atomic per cell and CTA
// instead of one per warp and cell), and hands out slots of those sub-ranges
// with shared-memory atomics.  Order inside a cell is unspecified.
template <typename PosT>
__global__ void k_sort_scatter_direct(Dev d, int s)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned int* cur_slot = (unsigned int*)smem_raw;          // [ncell]: count, then next slot
    __shared__ int s_last;
    const int N = d.ncell;
    const long long n = d.ctl->n[s];
    const unsigned int cur = d.ctl->cur[s];
    const SpBuf A = d.buf[s][cur], Bn = d.buf[s][cur ^ 1u];
    const PosT* PA = (const PosT*)A.pos;
    PosT* PB = (PosT*)Bn.pos;
    const int lane = threadIdx.x & 31;
    const long long i0 = n * blockIdx.x / gridDim.x, i1 = n * (blockIdx.x + 1) / gridDim.x;
    // all lanes of a warp run the same number of iterations (warp-wide collectives below)
    const long long i1r = i0 + (i1 - i0 + blockDim.x - 1) / blockDim.x * blockDim.x;
    for (int m = threadIdx.x; m < N; m += blockDim.x) cur_slot[m] = 0;
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        for (long long i = i0 + threadIdx.x; i < i1r; i += blockDim.x) {
            bool act = i < i1;
            PosT x = 0;
            float fx = 0.0f, fy = 0.0f, fz = 0.0f;
            uint64_t fid = 0;
            uint32_t fnev = 0;
            if (act) {
                x = PA[i];
                if (pass == 1) {                           // in flight while the slot is worked out
                    fx = A.vx[i];
                    fy = A.vy[i];
                    fz = A.vz[i];
                    fid = A.id[i];
                    fnev = A.nev[i];
                }
                act = is_alive(x);
            }
            uint32_t j = 0xffffffffu, wr;
            if (act) {
                cell_of(x, d.kshift, j, wr);
                if (j >= (uint32_t)N) {
                    act = false;
                    j = 0xffffffffu;
                }
            }
            // lanes of one cell share one shared-memory atomic (cell-sorted input would
            // otherwise serialise on a single counter)
            const unsigned grp = __match_any_sync(0xffffffffu, j);
            const int leader = __ffs(grp) - 1;
            const int rank = __popc(grp & ((1u << lane) - 1u));
            unsigned int base = 0;
            if (act && lane == leader) base = atomicAdd(&cur_slot[j], (unsigned)__popc(grp));
            if (pass == 0) continue;
            base = __shfl_sync(0xffffffffu, base, leader);
            if (act) {
                const unsigned int o = base + rank;
                PB[o] = x;
                Bn.vx[o] = fx;
                Bn.vy[o] = fy;
                Bn.vz[o] = fz;
                Bn.id[o] = fid;
                Bn.nev[o] = fnev;
            }
        }
        __syncthreads();
        if (pass == 0) {                                   // reserve this CTA's sub-range of every touched cell
            for (int m = threadIdx.x; m < N; m += blockDim.x) {
                const unsigned int c = cur_slot[m];
                if (c) cur_slot[m] = atomicAdd(&d.sort_off[m], c);
            }
            __syncthreads();
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

// Staged scatter (electrons and test particles, whose cell order is gone a
// few steps after a compaction): each CTA takes a contiguous run of slots,
// counts its particles per cell in shared memory, and reserves one sub-range
// per touched cell of the cell's global range (one global atomic per cell and
// CTA).  It then moves
// its run in chunks of kSortChunk particles: a counting sort of the chunk by
// cell in shared memory, then each cell's part of the chunk written as one
// contiguous run of its sub-range.  Scattering every particle straight from
// registers made one L2 write request per particle and array for cell-mixed
// input (electrons), which bounded the kernel; runs of several particles
// per cell share requests and fill whole sectors.  Order inside a cell is
// unspecified.
constexpr int kSortThreads = 1024;
#ifndef PG_SORT_PER
#define PG_SORT_PER 4
#endif
constexpr int kSortPer = PG_SORT_PER;                         // particles per thread and chunk
constexpr int kSortChunk = kSortThreads * kSortPer;
// shared memory at the largest case, 4096 cells and 64-bit positions, within the 227 KB a CTA may have
static_assert(4096 * 12 + (size_t)kSortChunk * (8 + 8 + 4 * 5) <= 227 * 1024, "staged sort chunk too large");
template <typename PosT>
size_t sort_scatter_smem_t(int ncell)
{
    return (size_t)ncell * 12 + (size_t)kSortChunk * (sizeof(PosT) + 8 + 4 * 5);
}
size_t sort_scatter_smem(int ncell, bool p64)
{
    return p64 ? sort_scatter_smem_t<double>(ncell) : sort_scatter_smem_t<uint32_t>(ncell);
}

template <typename PosT>
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter_staged(Dev d, int s)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = d.ncell;
    // [cur_slot u32 N][hc u32 N][ho u32 N][x PosT C][id u64 C][vx vy vz nev cell u32 C]
    unsigned int* cur_slot = (unsigned int*)smem_raw;        // this CTA's next slot of each cell
    unsigned int* hc = cur_slot + N;                          // the chunk's count per cell
    unsigned int* ho = hc + N;                                // the chunk's first staged entry per cell
    unsigned char* stg = smem_raw + (((size_t)N * 12 + 15) & ~(size_t)15);
    PosT* sx = (PosT*)stg;
    uint64_t* sid = (uint64_t*)(stg + (size_t)kSortChunk * sizeof(PosT));
    float* svx = (float*)(sid + kSortChunk);
    float* svy = svx + kSortChunk;
    float* svz = svy + kSortChunk;
    uint32_t* snev = (uint32_t*)(svz + kSortChunk);
    uint32_t* scell = snev + kSortChunk;
    __shared__ int s_last;
    __shared__ long long sh_scan[32];

    const long long n = d.ctl->n[s];
    const unsigned int cur = d.ctl->cur[s];
    const SpBuf A = d.buf[s][cur], Bn = d.buf[s][cur ^ 1u];
    const PosT* PA = (const PosT*)A.pos;
    PosT* PB = (PosT*)Bn.pos;
    const int lane = threadIdx.x & 31, T = blockDim.x;
    const long long i0 = n * blockIdx.x / gridDim.x, i1 = n * (blockIdx.x + 1) / gridDim.x;
    for (int m = threadIdx.x; m < N; m += T) {
        cur_slot[m] = 0;
        hc[m] = 0;
    }
    __syncthreads();

    // cell of slot i, or 0xffffffff for a removed slot
    auto cell_at = [&](PosT x) -> uint32_t {
        if (!is_alive(x)) return 0xffffffffu;
        uint32_t j, wr;
        cell_of(x, d.kshift, j, wr);
        return j < (uint32_t)N ? j : 0xffffffffu;
    };
    // lanes of one cell share one shared-memory atomic (cell-ordered input would
    // otherwise serialise on a single counter); returns the lane's rank
    auto add_count = [&](unsigned int* cnt, uint32_t j) -> unsigned int {
        const unsigned grp = __match_any_sync(0xffffffffu, j);
        const int leader = __ffs(grp) - 1;
        const unsigned int rank = __popc(grp & ((1u << lane) - 1u));
        unsigned int base = 0;
        if (j != 0xffffffffu && lane == leader) base = atomicAdd(&cnt[j], (unsigned)__popc(grp));
        return __shfl_sync(0xffffffffu, base, leader) + rank;
    };

    // 1. this CTA's particles per cell, then one sub-range of every touched cell
    const long long i1r = i0 + (i1 - i0 + T - 1) / T * T;     // whole warps: collectives above
    for (long long i = i0 + threadIdx.x; i < i1r; i += T) {
        const uint32_t j = i < i1 ? cell_at(PA[i]) : 0xffffffffu;
        add_count(cur_slot, j);
    }
    __syncthreads();
    for (int m = threadIdx.x; m < N; m += T) {
        const unsigned int c = cur_slot[m];
        if (c) cur_slot[m] = atomicAdd(&d.sort_off[m], c);
    }
    __syncthreads();

    // 2. the run in chunks: count by cell, stage in cell order, write each cell's part as one run
    const int seg = (N + T - 1) / T;                          // cells per thread in the scan
    const int m0 = min((int)threadIdx.x * seg, N), m1 = min(m0 + seg, N);
    for (long long c0 = i0; c0 < i1; c0 += kSortChunk) {
        PosT x[kSortPer];
        float fx[kSortPer], fy[kSortPer], fz[kSortPer];
        uint64_t fid[kSortPer];
        uint32_t fnev[kSortPer], jj[kSortPer], rk[kSortPer];
#pragma unroll
        for (int k = 0; k < kSortPer; ++k) {                  // all loads in flight together
            const long long i = c0 + threadIdx.x + (long long)k * T;
            x[k] = 0;
            fx[k] = fy[k] = fz[k] = 0.0f;
            fid[k] = 0;
            fnev[k] = 0;
            if (i < i1) {
                x[k] = PA[i];
                fx[k] = A.vx[i];
                fy[k] = A.vy[i];
                fz[k] = A.vz[i];
                fid[k] = A.id[i];
                fnev[k] = A.nev[i];
            }
        }
#pragma unroll
        for (int k = 0; k < kSortPer; ++k) {
            const long long i = c0 + threadIdx.x + (long long)k * T;
            jj[k] = i < i1 ? cell_at(x[k]) : 0xffffffffu;
            rk[k] = add_count(hc, jj[k]);
        }
        __syncthreads();
        long long a = 0;
        for (int m = m0; m < m1; ++m) a += hc[m];
        long long tot_l;
        long long off = block_exclusive_scan(a, sh_scan, tot_l);
        const unsigned int tot = (unsigned int)tot_l;
        for (int m = m0; m < m1; ++m) {
            ho[m] = (unsigned int)off;
            off += hc[m];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kSortPer; ++k) {
            if (jj[k] == 0xffffffffu) continue;
            const unsigned int p = ho[jj[k]] + rk[k];
            sx[p] = x[k];
            sid[p] = fid[k];
            svx[p] = fx[k];
            svy[p] = fy[k];
            svz[p] = fz[k];
            snev[p] = fnev[k];
            scell[p] = jj[k];
        }
        __syncthreads();
        for (unsigned int p = threadIdx.x; p < tot; p += T) {
            const uint32_t j = scell[p];
            const unsigned int o = cur_slot[j] + (p - ho[j]);
            PB[o] = sx[p];
            Bn.vx[o] = svx[p];
            Bn.vy[o] = svy[p];
            Bn.vz[o] = svz[p];
            Bn.id[o] = sid[p];
            Bn.nev[o] = snev[p];
        }
        __syncthreads();
        for (int m = threadIdx.x; m < N; m += T) {
            cur_slot[m] += hc[m];
            hc[m] = 0;
        }
        __syncthreads();
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
    return 2 * q_bytes16(ncell) + acc_bytes(ncell) + (size_t)ncell * 8 + (size_t)N1 * 4 + kNbEedf * 4 +
           kQueueCap * 4;
}

cudaError_t launch_init(const Dev& d, int s, long long n, long long id0, float vth, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int T = 256;
    const long long G = (n + T - 1) / T;
    if (d.pos64 && s != kTP) k_init<true><<<(unsigned)G, T, 0, st>>>(d, s, n, id0, vth);
    else k_init<false><<<(unsigned)G, T, 0, st>>>(d, s, n, id0, vth);
    return cudaGetLastError();
}

static cudaError_t set_smem_attr(const void* fn, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t mover_occupancy(const Dev& d, int* blocks_per_sm)
{
    const size_t sm = mover_smem(d.ncell);
    const void* fn = d.pos64 ? (const void*)k_mover<true, 0, false> : (const void*)k_mover<false, 0, false>;
    cudaError_t e = set_smem_attr(fn, sm);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kMoverThreads, sm);
}

template <bool P64>
static cudaError_t launch_mover_t(const Dev& d, const StepArgs& a, int grid, int mode, cudaStream_t st)
{
    const size_t sm = mover_smem(d.ncell);
    const bool sample = mode == 0 && d.diag_every > 0 && (a.step + 1u) % (unsigned)d.diag_every == 0;
    const void* fn = mode == 1 ? (const void*)k_mover<P64, 1, false>
                               : (sample ? (const void*)k_mover<P64, 0, true> : (const void*)k_mover<P64, 0, false>);
    cudaError_t e = set_smem_attr(fn, sm);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kMoverThreads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = kMoverPdl;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (mode == 1) return cudaLaunchKernelEx(&cfg, k_mover<P64, 1, false>, d, a);
    if (sample) return cudaLaunchKernelEx(&cfg, k_mover<P64, 0, true>, d, a);
    return cudaLaunchKernelEx(&cfg, k_mover<P64, 0, false>, d, a);
}

cudaError_t launch_mover_batch(const BatchEntry* ent, const int* owner, int grid, int max_ncell, bool sample,
                               cudaStream_t st)
{
    const size_t sm = mover_smem(max_ncell);      // attribute set by mover_batch_attr
    if (sample) k_mover_batch<true><<<grid, kMoverThreads, sm, st>>>(ent, owner);
    else k_mover_batch<false><<<grid, kMoverThreads, sm, st>>>(ent, owner);
    return cudaGetLastError();
}

cudaError_t launch_mover_batch_chunks(const BatchEntry* ent, const BatchChunk* chunks, int nchunks, unsigned int* work,
                                      int grid, int max_ncell, bool sample, cudaStream_t st)
{
    const size_t sm = mover_smem(max_ncell);      // attribute set by mover_batch_attr
    if (sample) k_mover_batch_chunks<true><<<grid, kMoverThreads, sm, st>>>(ent, chunks, nchunks, work);
    else k_mover_batch_chunks<false><<<grid, kMoverThreads, sm, st>>>(ent, chunks, nchunks, work);
    return cudaGetLastError();
}

cudaError_t mover_batch_attr(int max_ncell, int* blocks_per_sm)
{
    const size_t sm = mover_smem(max_ncell);
    cudaError_t e = set_smem_attr((const void*)k_mover_batch<true>, sm);
    if (e != cudaSuccess) return e;
    e = set_smem_attr((const void*)k_mover_batch_chunks<true>, sm);
    if (e != cudaSuccess) return e;
    e = set_smem_attr((const void*)k_mover_batch_chunks<false>, sm);
    if (e != cudaSuccess) return e;
    e = set_smem_attr((const void*)k_mover_batch<false>, sm);
    if (e != cudaSuccess || !blocks_per_sm) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, (const void*)k_mover_batch<false>,
                                                         kMoverThreads, sm);
}

cudaError_t launch_mover(const Dev& d, const StepArgs& a, int grid, int mode, cudaStream_t st)
{
    return d.pos64 ? launch_mover_t<true>(d, a, grid, mode, st) : launch_mover_t<false>(d, a, grid, mode, st);
}

cudaError_t launch_entry_nev(const Dev& d, int s, unsigned int half, long long n, unsigned int l0, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const long long b = (n + 255) / 256;
    k_entry_nev<<<(int)(b < 4096 ? b : 4096), 256, 0, st>>>(d, s, half, n, l0);
    return cudaGetLastError();
}

cudaError_t launch_sort(const Dev& d, int s, int grid, cudaStream_t st)
{
    const bool p64 = d.pos64 && s != kTP;
    const size_t sm = (size_t)d.ncell * 4;
    const int gs = grid >= 8 ? grid / 4 : grid;     // longer runs per CTA: fewer cell reservations
    if (p64) k_sort_count<double><<<gs, 1024, sm, st>>>(d, s);
    else k_sort_count<uint32_t><<<gs, 1024, sm, st>>>(d, s);
    k_sort_scan<<<1, 1024, 0, st>>>(d);
    if (s == kI) {                                  // cell-ordered: stores are runs already
        if (p64) k_sort_scatter_direct<double><<<gs, 1024, sm, st>>>(d, s);
        else k_sort_scatter_direct<uint32_t><<<gs, 1024, sm, st>>>(d, s);
        return cudaGetLastError();
    }
    // cell-mixed: the staged scatter on its resident CTAs (one or two per SM, by its shared memory)
    const size_t ss = sort_scatter_smem(d.ncell, p64);
    const void* fn = p64 ? (const void*)k_sort_scatter_staged<double> : (const void*)k_sort_scatter_staged<uint32_t>;
    cudaError_t e = set_smem_attr(fn, ss);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSortThreads, ss);
    if (e != cudaSuccess) return e;
    const int gsc = std::max(1, (grid >= 8 ? grid / 8 : 1) * std::max(per_sm, 1));
    if (p64) k_sort_scatter_staged<double><<<gsc, kSortThreads, ss, st>>>(d, s);
    else k_sort_scatter_staged<uint32_t><<<gsc, kSortThreads, ss, st>>>(d, s);
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

cudaError_t launch_field(const Dev& d, double v_left, int accumulate, cudaStream_t st)
{
    k_field<<<1, 512, 0, st>>>(d, v_left, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_op_poisson(const long long* qi, const long long* qe, int N, double A, double inv_dx,
                              double v_left, double* phi, double* E64, cudaStream_t st)
{
    k_op_poisson<<<1, 512, 0, st>>>(qi, qe, N, A, inv_dx, v_left, phi, E64);
    return cudaGetLastError();
}

}  // namespace pg
