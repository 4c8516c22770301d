// tp_kernels.cu -- test-particle transport of sputtered Al atoms (sm_103a).
//
// Sec. "Test Particle Method" of arXiv:1607.04069: every atom is traced with
// a fixed step, x += v_x dt; it sticks to either electrode (perfect sink,
// absorbed flux recorded); otherwise it meets a thermal Ar partner w with
// probability 1 - exp(-n sigma |v - w| dt) (Eq. collisionprobability1 with
// tau_c = 1/(n sigma g)) and scatters isotropically in the centre-of-mass
// frame (hard sphere).  No feedback onto the plasma.
#include "common.cuh"
#include "launch.h"
#include "solve.cuh"

namespace pg {

// Tallies of one CTA's tile on sample steps: the deposit as 32-bit counters
// (atoms n_j, high and low 16 bits of their right-node weights, as in the
// step kernel) and the v_x moment as 64-bit sums kept in (low, high) 32-bit
// pairs -- 64-bit shared atomics are not native.  With at most 65536 atoms
// per tile no counter can overflow.
constexpr long long kTpTileGroups = 16384;   // 65536 atoms
struct TpAcc {
    unsigned int *cnt, *whi, *wlo;   // [N]
    unsigned int* flo;               // [N+1]
    int* fhi;                        // [N+1]
};

__device__ __forceinline__ void tp_add64(const TpAcc& A, int m, long long v)
{
    const unsigned int vl = (unsigned int)v;
    const unsigned int old = atomicAdd(&A.flo[m], vl);
    const int vh = (int)(v >> 32) + (old + vl < old ? 1 : 0);
    if (vh) atomicAdd(&A.fhi[m], vh);
}

__device__ void tp_flush(const TpAcc& A, int N, unsigned long long* q, long long* f, int t, int nt)
{
    for (int m = t; m <= N; m += nt) {
        unsigned long long v = 0;
        if (m < N) v += ((unsigned long long)A.cnt[m] << 32) - (((unsigned long long)A.whi[m] << 16) + A.wlo[m]);
        if (m > 0) v += ((unsigned long long)A.whi[m - 1] << 16) + A.wlo[m - 1];
        if (v) atomicAdd(&q[m], v);
        const long long fv = (long long)(((unsigned long long)(unsigned int)A.fhi[m] << 32) | A.flo[m]);
        if (fv) atomicAdd((unsigned long long*)&f[m], (unsigned long long)fv);
    }
    __syncthreads();                                   // node m also reads cell m-1: clear after all reads
    for (int m = t; m <= N; m += nt) {
        if (m < N) A.cnt[m] = A.whi[m] = A.wlo[m] = 0;
        A.flo[m] = 0;
        A.fhi[m] = 0;
    }
}

// A run of consecutive atoms of one lane in cell j, summed as the shared
// tallies are (per-lane sums stay below the tallies' 65536-atom span bound).
constexpr uint32_t kTpNoRun = 0xffffffffu;
struct TpRun {
    uint32_t j, cnt = 0, whi = 0, wlo = 0;
    long long f0 = 0, f1 = 0;    // flux moment at nodes j and j+1
};
__device__ __forceinline__ void tp_run_flush(const TpAcc& A, TpRun& r)
{
    if (r.j == kTpNoRun) return;
    atomicAdd(&A.cnt[r.j], r.cnt);
    atomicAdd(&A.whi[r.j], r.whi);
    atomicAdd(&A.wlo[r.j], r.wlo);
    if (r.f0) tp_add64(A, (int)r.j, r.f0);
    if (r.f1) tp_add64(A, (int)r.j + 1, r.f1);
    r.cnt = r.whi = r.wlo = 0;
    r.f0 = r.f1 = 0;
}

struct TpGrp {                 // one group of four atoms, as loaded
    uint4 P;
    float4 VX, VY, VZ;
    ulonglong2 Ia, Ib;
};
__device__ __forceinline__ TpGrp tp_load(const SpBuf& B, long long g)
{
    TpGrp G;
    G.P = ((const uint4*)B.pos)[g];
    G.VX = ((const float4*)B.vx)[g];
    G.VY = ((const float4*)B.vy)[g];
    G.VZ = ((const float4*)B.vz)[g];
    G.Ia = ((const ulonglong2*)B.id)[2 * g];
    G.Ib = ((const ulonglong2*)B.id)[2 * g + 1];
    return G;
}

// One TP step.  Atoms are taken in groups of four (16-byte vector loads of x
// and v, 32 bytes of ids); each CTA owns a contiguous run of groups.  The two
// Philox blocks of every atom (gas partner, collision test) are drawn for the
// four atoms of a group at once, their rounds interleaved.
// Collision law of the TP kernels (Sec. "Binary Interactions"): the per-step
// rate n sigma(g) g dt, for hard spheres n sigma_tp g dt and for the VHS and
// M1 laws n K g^alpha dt.
template <bool LAW>
__device__ __forceinline__ float tp_rate_dt(const Dev& d, float nsig_dt, float nK_dt, float g)
{
    return LAW ? nK_dt * powf(g, d.tp_alpha) : nsig_dt * g;
}

// Direction of the post-collision relative velocity: isotropic for hard
// spheres and VHS; M1 turns g by chi = pi (1 - sqrt(r1)) at the azimuth
// 2 pi r2 about g (frame: e1 along g x x^, or g x y^ when |g_x| >= 0.9 |g|,
// e2 = g^ x e1).
__device__ __forceinline__ float3 tp_scatter_dir(int model, float gx, float gy, float gz, float gm, uint32_t r1, uint32_t r2)
{
    if (model != 2 || gm == 0.0f) return iso_dir(r1, r2);
    const float ux = gx / gm, uy = gy / gm, uz = gz / gm;
    const bool xa = fabsf(ux) < 0.9f;
    // e1 = u x a with a = x^ or y^
    float e1x = xa ? 0.0f : -uz, e1y = xa ? uz : 0.0f, e1z = xa ? -uy : ux;
    const float n1 = sqrtf(e1x * e1x + e1y * e1y + e1z * e1z);
    e1x /= n1; e1y /= n1; e1z /= n1;
    const float e2x = uy * e1z - uz * e1y, e2y = uz * e1x - ux * e1z, e2z = ux * e1y - uy * e1x;
    float sc, cc, se, ce;                       // chi = pi (1 - sqrt(r1)), eps = 2 pi r2
    sincospif(1.0f - sqrtf(u23(r1)), &sc, &cc);
    sincospif(2.0f * u23(r2), &se, &ce);
    return make_float3(cc * ux + sc * (ce * e1x + se * e2x), cc * uy + sc * (ce * e1y + se * e2y),
                       cc * uz + sc * (ce * e1z + se * e2z));
}

// The fixed-point move of one TP step: the new position, or the electrode
// reached (0 at x = 0, 1 at x = L; -1 inside).  The displacement rint(v_x dt
// 2^32 / L) is converted to 32 bits and the exit is a wrap-around test, as in
// the step kernel; 64-bit integer conversions run on the FP64 units, which
// this part has few of.  A displacement beyond +-2^31 units (far more than a
// step of any realistic atom) takes the 64-bit form.
__device__ __forceinline__ int tp_move(uint32_t x, float vx, float scale, uint32_t* xn)
{
    const float fd = vx * scale;
    if (fabsf(fd) < 2147483520.0f) {
        const int disp = __float2int_rn(fd);
        const uint32_t xm = x + (uint32_t)disp;
        if (disp > 0 && xm < x) return 1;
        if (disp < 0 && (0u - (uint32_t)disp) >= x) return 0;
        *xn = xm;
        return -1;
    }
    const long long np = (long long)x + __float2ll_rn(fd);
    if (np <= 0) return 0;
    if (np >= 4294967296LL) return 1;
    *xn = (uint32_t)np;
    return -1;
}

// LAW: the VHS / M1 laws (tp_model 1, 2); else hard spheres
template <bool LAW>
__global__ void __launch_bounds__(kTpThreads, 2) k_tp_step(Dev d)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = d.ncell;
    TpAcc A;
    A.cnt = (unsigned int*)smem_raw;
    A.whi = A.cnt + N;
    A.wlo = A.whi + N;
    A.flo = A.wlo + N;
    A.fhi = (int*)(A.flo + N + 1);
    __shared__ unsigned int s_coll;
    __shared__ int s_last;

    Ctl* ctl = d.ctl;
    const unsigned int s = ctl->tp_step;
    const long long n = ctl->n[kTP];
    const bool sample = d.diag_every > 0 && ((s + 1) % (unsigned)d.diag_every == 0);
    const long long G4 = (n + 3) >> 2;
    const long long g0 = G4 * blockIdx.x / gridDim.x, g1 = G4 * (blockIdx.x + 1) / gridDim.x;
    if (sample)
        for (int m = threadIdx.x; m <= N; m += blockDim.x) {
            if (m < N) A.cnt[m] = A.whi[m] = A.wlo[m] = 0;
            A.flo[m] = 0;
            A.fhi[m] = 0;
        }
    if (threadIdx.x == 0) s_coll = 0;
    __syncthreads();

    const SpBuf B = d.buf[kTP][ctl->cur[kTP]];
    const float mu_al = (float)(kMAL / (kMAL + kMAR)), mu_ar = (float)(kMAR / (kMAL + kMAR));
    const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
    unsigned int ncoll = 0;
    for (long long t0 = g0; t0 < g1; t0 += kTpTileGroups) {
        const long long t1 = min(g1, t0 + kTpTileGroups);
        // each thread loads its next group before working on the current one
        long long g = t0 + threadIdx.x;
        TpGrp nxt;
        if (g < t1) nxt = tp_load(B, g);
        for (; g < t1; g += blockDim.x) {
            const TpGrp cur = nxt;
            if (g + blockDim.x < t1) nxt = tp_load(B, g + blockDim.x);
            uint32_t x[4] = {cur.P.x, cur.P.y, cur.P.z, cur.P.w};
            if (4 * g + 4 > n)                             // slots past n hold no atom
#pragma unroll
                for (int u = 1; u < 4; ++u)
                    if (4 * g + u >= n) x[u] = 0u;
            if ((x[0] | x[1] | x[2] | x[3]) == 0u) continue;
            const float4 VX = cur.VX, VY = cur.VY, VZ = cur.VZ;
            const ulonglong2 Ia = cur.Ia, Ib = cur.Ib;
            float vx[4] = {VX.x, VX.y, VX.z, VX.w}, vy[4] = {VY.x, VY.y, VY.z, VY.w}, vz[4] = {VZ.x, VZ.y, VZ.z, VZ.w};
            const uint64_t id[4] = {Ia.x, Ia.y, Ib.x, Ib.y};
            uint4 cg[4], cc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                cg[u] = make_uint4((uint32_t)id[u], (uint32_t)(id[u] >> 32), s, kPurTpGas);
                cc[u] = make_uint4((uint32_t)id[u], (uint32_t)(id[u] >> 32), s, kPurTpColl);
            }
            philox_n<4>(cg, k0, k1);
            philox_n<4>(cc, k0, k1);
            bool moved = false;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (x[u] == 0u) continue;
                uint32_t xm = 0u;
                const int el = tp_move(x[u], vx[u], d.tp_scale, &xm);
                if (el >= 0) {                              // sticks at an electrode
                    const float v2 = vx[u] * vx[u] + vy[u] * vy[u] + vz[u] * vz[u];
                    const float E = v2 * (float)(0.5 * kMAL / kQE);
                    const float ct = fminf(v2 > 0.0f ? fabsf(vx[u]) * rsqrtf(v2) : 1.0f, 1.0f);
                    const int be = hist_bin(E, 300.0f, kNbSpE);
                    const int ba = clamp_bin(acosf(ct) * (float)(180.0 / kPI), kNbAng);
                    atomicAdd(&d.diag.sp_e[el][be], 1ull);
                    atomicAdd(&d.diag.sp_ang[el][ba], 1ull);
                    atomicAdd(&ctl->cnt[el == 0 ? kCntTpDepL : kCntTpDepR], 1ull);
                    x[u] = 0u;
                    continue;
                }
                x[u] = xm;
                // Collision test u < Pc(g), Pc = 1 - exp(-n sigma g dt), g = |v - w| for the gas
                // partner w of this step.  First against an upper bound of g that needs only the
                // Box-Muller radii (n1^2 + n2^2 = r1^2, n3^2 <= r2^2): most atoms fail it, and the
                // partner's directions and the exact g are then not needed.  The bound carries a
                // relative margin of 1e-4 over the FP32 roundings, so it never rejects an atom
                // that the exact test below would accept.
                const float uc = u23(cc[u].x);
                const float r1s = -2.0f * logf(u23(cg[u].x)), r2s = -2.0f * logf(u23(cg[u].z));
                const float vm = sqrtf(vx[u] * vx[u] + vy[u] * vy[u] + vz[u] * vz[u]);
                const float gub = 1.0001f * (vm + d.vth_gas * sqrtf(r1s + r2s));
                if (uc < -expm1f(-tp_rate_dt<LAW>(d, d.tp_nsig_dt, d.tp_nK_dt, gub))) {
                    const float2 n12 = box_muller(cg[u].x, cg[u].y);
                    const float2 n34 = box_muller(cg[u].z, cg[u].w);
                    const float wx = d.vth_gas * n12.x, wy = d.vth_gas * n12.y, wz = d.vth_gas * n34.x;
                    const float gx = vx[u] - wx, gy = vy[u] - wy, gz = vz[u] - wz;
                    const float gm = sqrtf(gx * gx + gy * gy + gz * gz);
                    const float Pc = -expm1f(-tp_rate_dt<LAW>(d, d.tp_nsig_dt, d.tp_nK_dt, gm));
                    if (uc < Pc) {                             // scattering in the centre of mass
                        const float3 dir = LAW ? tp_scatter_dir(d.tp_model, gx, gy, gz, gm, cc[u].y, cc[u].z)
                                               : iso_dir(cc[u].y, cc[u].z);
                        vx[u] = mu_al * vx[u] + mu_ar * wx + mu_ar * gm * dir.x;
                        vy[u] = mu_al * vy[u] + mu_ar * wy + mu_ar * gm * dir.y;
                        vz[u] = mu_al * vz[u] + mu_ar * wz + mu_ar * gm * dir.z;
                        moved = true;
                        ++ncoll;
                    }
                }
                if (sample) {
                    uint32_t j, wr;
                    cell_of(x[u], d.kshift, j, wr);
                    atomicAdd(&A.cnt[j], 1u);
                    atomicAdd(&A.whi[j], wr >> 16);
                    atomicAdd(&A.wlo[j], wr & 0xffffu);
                    const long long vq = (long long)__float2int_rn(vx[u]);
                    const long long w16 = (long long)(wr >> 16);
                    tp_add64(A, j, vq * (65536 - w16));
                    tp_add64(A, j + 1, vq * w16);
                }
            }
            ((uint4*)B.pos)[g] = make_uint4(x[0], x[1], x[2], x[3]);
            if (moved) {
                ((float4*)B.vx)[g] = make_float4(vx[0], vx[1], vx[2], vx[3]);
                ((float4*)B.vy)[g] = make_float4(vy[0], vy[1], vy[2], vy[3]);
                ((float4*)B.vz)[g] = make_float4(vz[0], vz[1], vz[2], vz[3]);
            }
        }
        if (sample) {                                      // this tile's tallies into the step's histograms
            __syncthreads();
            tp_flush(A, N, d.tp_q, d.tp_flux, threadIdx.x, blockDim.x);
            __syncthreads();
        }
    }
    ncoll = __reduce_add_sync(0xffffffffu, ncoll);
    if ((threadIdx.x & 31) == 0 && ncoll) atomicAdd(&s_coll, ncoll);
    __syncthreads();
    if (threadIdx.x == 0 && s_coll) atomicAdd(&ctl->cnt[kCntTpColl], (unsigned long long)s_coll);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ctl->tp_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int m = threadIdx.x; m <= N; m += blockDim.x) {
        if (sample) {
            red_split(d.diag.tp_dens + 2 * m, __ldcg(d.tp_q + m));
            red_split_signed(d.diag.tp_vx + 2 * m, __ldcg(d.tp_flux + m));
        }
        d.tp_q[m] = 0;
        d.tp_flux[m] = 0;
    }
    if (threadIdx.x == 0) {
        ctl->tp_step = s + 1;
        if (sample) ctl->n_tp_samp += 1;
        ctl->tp_done = 0;
    }
}


// ---------------------------------------------------------------- TP step, thinned candidates
// tp_mode 0 (Sec. "Test Particle Method", Eq. collisionprobability1 with a
// partner w from the Maxwellian gas): the per-step probability p(g) = 1 -
// exp(-n K dt g^alpha) (hard spheres: K = sigma_tp, alpha = 1) is bounded by
// n K dt (|v|^alpha + |w|^alpha) (alpha <= 1), so every step is a candidate
// with P^ = n K dt (|v|^alpha + <|w|^alpha>), rounded up to 8 significant
// bits; the steps between candidates are geometric and each atom keeps its
// next candidate step plus one in nev (0: none drawn yet, drawn at the first
// step that moves it).  A candidate draws one partner from (|v|^alpha +
// |w|^alpha) f(w) and collides with probability p(g) (|v|^alpha +
// <|w|^alpha>) / (P^ (|v|^alpha + |w|^alpha)); the product is f(w) p(g), the
// per-step law, and |v| changes only at a collision.  The stream thus reads
// x, v_x and the candidate step and writes x; v_y, v_z and the id are read
// only at candidates and at the walls.  Random words: (id, s, TP_GAP0) for the
// first gap, (id, s, TP_CAND / TP_CAND + 1) for the proposal, (id, s,
// TP_GAMMA + t) for its gamma attempts (VHS / M1), (id, s, TP_COLL) words 1, 2
// for the scattering, (id, s, TP_GAP) for the next gap; s the TP step.

// x rounded up to 8 significant bits (0, NaN and infinity unchanged)
__device__ __forceinline__ float round_up8(float x)
{
    if (!(x > 0.0f) || isinf(x)) return x;
    int e;
    const float m = frexpf(x, &e);
    return ldexpf(ceilf(m * 256.0f) * (1.0f / 256.0f), e);
}

// TP steps from one candidate to the next at the per-step probability Ph:
// 1 + floor(ln R / ln(1 - Ph)), the floor of the FP64 quotient; FP32 first,
// FP64 when an integer lies within the FP32 error of the quotient.
__device__ __noinline__ uint32_t tp_gap(float Ph, uint32_t w)
{
    if (!(Ph < 1.0f)) return 1u;
    if (!(Ph > 0.0f)) return 2147483647u;
    const float uf = u23(w);
    const float xf = logf(uf) / log1pf(-Ph);
    if (xf < 1.0e6f) {
        const float dl = 8e-7f * xf + 1e-6f;
        const float a = floorf(xf - dl), b = floorf(xf + dl);
        if (a == b) return 1u + (uint32_t)a;
    }
    const double x = log(((double)(w >> 9) + 0.5) * 0x1p-23) / log1p(-(double)Ph);
    if (!(x < 2147483646.0)) return 2147483647u;
    return 1u + (uint32_t)floor(x);
}

// the per-step candidate probability P^ of an atom of speed vm
template <bool LAW>
__device__ __forceinline__ float tp_cand_prob(const Dev& d, float vm)
{
    return LAW ? round_up8(d.tp_nK_dt * (powf(vm, d.tp_alpha) + d.tp_ma))
               : round_up8(d.tp_nsig_dt * (vm + d.tp_ma));
}

// Gamma variate of shape k >= 1 (Marsaglia and Tsang, ACM TOMS 26, 2000),
// attempt t from Philox(id, ctr, base + t); d after 32 rejections
__device__ __noinline__ float gamma_mt(float k, uint64_t seed, uint64_t id, uint32_t ctr, uint32_t base)
{
    const float dd = k - (1.0f / 3.0f), cc = 1.0f / sqrtf(9.0f * dd);
    for (int t = 0; t < 32; ++t) {
        const uint4 r = draw(seed, id, ctr, base + t);
        const float x = box_muller(r.x, r.y).x;
        float v = 1.0f + cc * x;
        if (v <= 0.0f) continue;
        v = v * v * v;
        if (logf(u23(r.z)) < 0.5f * x * x + dd - dd * v + dd * logf(v)) return dd * v;
    }
    return dd;
}

// An atom whose candidate step is due (or not drawn yet) at TP step s: draws
// the first gap if needed, handles the candidate and draws the next gap.
// Returns the new v_x; v_y, v_z and nev are stored here.  *hit: a collision.
template <bool LAW>
__device__ __noinline__ float tp_candidate(const Dev& d, const SpBuf& B, long long i, uint32_t s, float vx,
                                           uint32_t nv, bool* hit)
{
    float vy = B.vy[i], vz = B.vz[i];
    const uint64_t id = B.id[i];
    const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
    float vm = sqrtf(vx * vx + vy * vy + vz * vz);
    *hit = false;
    if (nv == 0u || (int)(nv - 1u - s) < 0) {                 // first gap of this atom
        const float Ph = tp_cand_prob<LAW>(d, vm);
        if (!(Ph <= 1.0f)) atomicAdd(&d.ctl->cnt[kCntNumerics], 1ull);
        nv = s + tp_gap(Ph, draw(d.seed, id, s, kPurTpGap0).x);
    }
    if (nv - 1u != s) {
        B.nev[i] = nv;
        return vx;
    }
    uint4 cw[2];
    cw[0] = make_uint4((uint32_t)id, (uint32_t)(id >> 32), s, kPurTpCand);
    cw[1] = make_uint4((uint32_t)id, (uint32_t)(id >> 32), s, kPurTpCand + 1);
    philox_n<2>(cw, k0, k1);
    const uint4 a = cw[0], b = cw[1];
    const float c = d.tpf_c;
    const float va = LAW ? powf(vm, d.tp_alpha) : vm;
    float wx, wy, wz;
    if (u23(a.x) * (va + d.tp_ma) < va) {                    // a Maxwellian partner
        const float2 n12 = box_muller(a.y, a.z), n34 = box_muller(a.w, b.x);
        wx = d.vth_gas * n12.x; wy = d.vth_gas * n12.y; wz = d.vth_gas * n34.x;
    } else {                                                 // |w|^alpha-weighted partner
        const float x2 = LAW ? gamma_mt(d.tpf_gk, d.seed, id, s, kPurTpGamma) : -logf(u23(a.y) * u23(a.z));
        const float sp = c * sqrtf(x2);
        const float3 dd = iso_dir(a.w, b.x);
        wx = sp * dd.x; wy = sp * dd.y; wz = sp * dd.z;
    }
    const float gx = vx - wx, gy = vy - wy, gz = vz - wz;
    const float gm = sqrtf(gx * gx + gy * gy + gz * gz);
    const float wm = sqrtf(wx * wx + wy * wy + wz * wz);
    const float Ph = tp_cand_prob<LAW>(d, vm);
    const float ga = LAW ? powf(gm, d.tp_alpha) : gm, wa = LAW ? powf(wm, d.tp_alpha) : wm;
    const float bK = LAW ? d.tp_nK_dt : d.tp_nsig_dt;
    if (u23(b.y) * Ph * (va + wa) < (va + d.tp_ma) * -expm1f(-bK * ga)) {   // a real collision
        const uint4 cc = draw(d.seed, id, s, kPurTpColl);
        const float3 dir = LAW ? tp_scatter_dir(d.tp_model, gx, gy, gz, gm, cc.y, cc.z) : iso_dir(cc.y, cc.z);
        const float mu_al = (float)(kMAL / (kMAL + kMAR)), mu_ar = (float)(kMAR / (kMAL + kMAR));
        vx = mu_al * vx + mu_ar * wx + mu_ar * gm * dir.x;
        vy = mu_al * vy + mu_ar * wy + mu_ar * gm * dir.y;
        vz = mu_al * vz + mu_ar * wz + mu_ar * gm * dir.z;
        B.vy[i] = vy;
        B.vz[i] = vz;
        vm = sqrtf(vx * vx + vy * vy + vz * vz);
        *hit = true;
    }
    const float Pn = tp_cand_prob<LAW>(d, vm);
    if (!(Pn <= 1.0f)) atomicAdd(&d.ctl->cnt[kCntNumerics], 1ull);
    B.nev[i] = s + 1u + tp_gap(Pn, draw(d.seed, id, s, kPurTpGap).x);
    return vx;
}

// An atom that reached an electrode: its energy and angle into that
// electrode's deposition histograms (Sec. "Wall Interactions" of the TPM)
__device__ __noinline__ void tp_stick(const Dev& d, const SpBuf& B, long long i, int el, float vx)
{
    const float vy = B.vy[i], vz = B.vz[i];
    const float v2 = vx * vx + vy * vy + vz * vz;
    const float E = v2 * (float)(0.5 * kMAL / kQE);
    const float ct = fminf(v2 > 0.0f ? fabsf(vx) * rsqrtf(v2) : 1.0f, 1.0f);
    atomicAdd(&d.diag.sp_e[el][hist_bin(E, 300.0f, kNbSpE)], 1ull);
    atomicAdd(&d.diag.sp_ang[el][clamp_bin(acosf(ct) * (float)(180.0 / kPI), kNbAng)], 1ull);
    atomicAdd(&d.ctl->cnt[el == 0 ? kCntTpDepL : kCntTpDepR], 1ull);
}

// The stream of the thinned-candidate TP step is staged in shared memory by
// bulk copies, one pipeline per warp: the CTA's contiguous run of 4-atom
// groups is cut into tiles of 64 groups (two per lane), which the warps
// claim one at a time from a shared counter (a warp slowed by a rare
// candidate takes fewer), and lane 0 keeps the next tile's x, v_x and
// candidate-step arrays (3 x 1 KB per tile) in flight in a ring of two
// stages, each with its own mbarrier (100M atoms, tallies in every launch:
// 345 us per step, against 416 us with 32-group tiles in four stages and
// 364 us with one group per thread loaded ahead into registers).  Warps do not wait for one another,
// so a lane busy with a rare candidate holds up only its own warp.  x is
// stored back from registers; v_x only where a group's atom collided.
// Sample steps cut the run into spans of 16384 groups (65536 atoms, the
// limit of the 32-bit shared tallies) and flush the tallies between spans.
#ifndef PG_TP_WARP_TILE
#define PG_TP_WARP_TILE 64
#endif
#ifndef PG_TP_STAGES
#define PG_TP_STAGES 2
#endif
constexpr int kTpWarpTile = PG_TP_WARP_TILE;             // groups per warp tile
constexpr int kTpLaneGroups = kTpWarpTile / 32;          // groups per lane and tile
constexpr int kTpMaxStages = PG_TP_STAGES;

// stages per warp: half as many above 1024 cells, whose tallies take more shared memory
__host__ __device__ __forceinline__ int tp_stages(int N)
{
    return N <= 1024 ? kTpMaxStages : (kTpMaxStages > 1 ? kTpMaxStages / 2 : 1);
}
__host__ __device__ __forceinline__ size_t tp_tally_bytes128(int N)
{
    return (((size_t)N * 12 + (size_t)(N + 1) * 8) + 127) & ~(size_t)127;
}
// the warps' rings alone (steps that take no samples), and with the tallies after them
__host__ __device__ __forceinline__ size_t tp_ring_smem(int N)
{
    return (size_t)(kTpThreads / 32) * tp_stages(N) * 3 * kTpWarpTile * 16;
}
size_t tp_geo_smem(int N) { return tp_ring_smem(N) + tp_tally_bytes128(N); }

// SAMPLE: this step adds to the time averages.  The host picks the
// instantiation from its own count of TP steps, which the last CTA's increment
// of ctl->tp_step mirrors; only a sample launch carries the tallies in its
// shared memory (the others hold the rings alone and leave the L1 part of the
// SM's on-chip memory larger).  A sample launch sums each lane's consecutive
// atoms of one cell in registers and adds the run to the shared tallies when
// the cell changes: sputtered atoms crowd into a few cells near the electrodes,
// where per-atom shared atomics on one address serialise.
template <bool LAW, bool SAMPLE>
__global__ void __launch_bounds__(kTpThreads, kTpMinBlocks) k_tp_step_geo(Dev d)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = d.ncell;
    TpAcc A;                                                 // after the rings (sample launches only)
    A.cnt = (unsigned int*)(smem_raw + tp_ring_smem(N));
    A.whi = A.cnt + N;
    A.wlo = A.whi + N;
    A.flo = A.wlo + N;
    A.fhi = (int*)(A.flo + N + 1);
    __shared__ __align__(8) uint64_t s_bar[kTpThreads / 32][kTpMaxStages];
    __shared__ unsigned int s_coll, s_tile;
    __shared__ int s_last;

    Ctl* ctl = d.ctl;
    const unsigned int s = ctl->tp_step;
    const long long n = ctl->n[kTP];
    constexpr bool sample = SAMPLE;
    const long long G4 = (n + 3) >> 2;
    const long long g0 = G4 * blockIdx.x / gridDim.x, g1 = G4 * (blockIdx.x + 1) / gridDim.x;
    const SpBuf B = d.buf[kTP][ctl->cur[kTP]];
    const int S = tp_stages(N);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr unsigned kArr = kTpWarpTile * 16u;                // bytes per array of a tile
    unsigned char* ring = smem_raw + (size_t)wid * S * 3 * kArr;   // 16-byte aligned
    uint64_t* bars = s_bar[wid];
    if (sample)
        for (int m = threadIdx.x; m <= N; m += blockDim.x) {
            if (m < N) A.cnt[m] = A.whi[m] = A.wlo[m] = 0;
            A.flo[m] = 0;
            A.fhi[m] = 0;
        }
    if (threadIdx.x == 0) {
        s_coll = 0;
        s_tile = 0;
    }
    if (lane == 0) {
        for (int q = 0; q < S; ++q) mbar_init(&bars[q], 1);
        mbar_init_fence();
    }
    __syncthreads();

    // tile t of the span [t0, t1) into stage st
    auto issue = [&](long long t0, long long t1, int t, int st) {
        const long long gs = t0 + (long long)t * kTpWarpTile;
        const unsigned bytes = (unsigned)(min((long long)kTpWarpTile, t1 - gs) * 16);
        unsigned char* buf = ring + (size_t)st * 3 * kArr;
        uint64_t* bar = &bars[st];
        mbar_expect_tx(bar, 3 * bytes);
        bulk_g2s(buf, (const uint4*)B.pos + gs, bytes, bar);
        bulk_g2s(buf + kArr, (const float4*)B.vx + gs, bytes, bar);
        bulk_g2s(buf + 2 * kArr, (const uint4*)B.nev + gs, bytes, bar);
    };

    // the test of the bounded wait: one warp issues no copies, so its first
    // wait runs out with nothing in flight (pic_test_wait_timeout)
    const bool no_copies = d.tp_wait_test && blockIdx.x == 0 && wid == 0;
    unsigned int ncoll = 0;
    TpRun run;                                              // this lane's pending run of one cell
    run.j = kTpNoRun;
    unsigned int phase[kTpMaxStages];                       // waits completed on each stage's barrier
#pragma unroll
    for (int st = 0; st < kTpMaxStages; ++st) phase[st] = 0;
    bool dead = false;                                      // a wait gave up: this warp skips the rest
    const long long span = sample ? kTpTileGroups : (g1 - g0);
    for (long long t0 = g0; t0 < g1; t0 += span) {
        const long long t1 = min(g1, t0 + span);
        const int ntile = (int)((t1 - t0 + kTpWarpTile - 1) / kTpWarpTile);
        // the warp claims the span's tiles one at a time from the CTA's counter, so
        // that a warp slowed by rare candidates takes fewer; lane 0 claims and issues
        auto claim = [&](int st) -> int {
            int t = -1;
            if (lane == 0 && !dead) {
                const unsigned c = atomicAdd(&s_tile, 1u);
                if (c < (unsigned)ntile) {
                    t = (int)c;
                    if (!no_copies) issue(t0, t1, t, st);
                }
            }
            return __shfl_sync(0xffffffffu, t, 0);
        };
        int tile[kTpMaxStages];
        if (lane == 0) async_proxy_fence();                  // the previous span's reads of the ring are done
#pragma unroll
        for (int st = 0; st < kTpMaxStages; ++st) tile[st] = st < S ? claim(st) : -1;
        for (int st = 0;; st = st + 1 < S ? st + 1 : 0) {
            if (tile[st] < 0) {                              // claims only grow: empty stages stay empty
                bool any = false;
#pragma unroll
                for (int u = 0; u < kTpMaxStages; ++u) any |= tile[u] >= 0;
                if (!any) break;
                continue;
            }
            const bool ok = mbar_wait(&bars[st], phase[st] & 1u, d.tp_wait_spin);
            if (__any_sync(0xffffffffu, !ok)) {             // let this warp's copies in flight land, then stop
                if (lane == 0) {
                    atomicOr(&ctl->err, kErrTimeout);
                    if (!no_copies)
#pragma unroll
                        for (int u = 0; u < kTpMaxStages; ++u)
                            if (tile[u] >= 0) mbar_wait(&bars[u], phase[u] & 1u, d.tp_wait_spin);
                }
                __syncwarp();
                dead = true;
                break;
            }
            ++phase[st];
            const long long gs = t0 + (long long)tile[st] * kTpWarpTile;
            const unsigned char* buf = ring + (size_t)st * 3 * kArr;
#pragma unroll 1
            for (int r = 0; r < kTpLaneGroups; ++r) {
                const int e = lane + 32 * r;
                if (gs + e >= t1) break;
                const long long g = gs + e;
                const uint4 P = ((const uint4*)buf)[e];
                const float4 VX = ((const float4*)(buf + kArr))[e];
                const uint4 NV = ((const uint4*)(buf + 2 * kArr))[e];

                uint32_t x[4] = {P.x, P.y, P.z, P.w};
                float vx[4] = {VX.x, VX.y, VX.z, VX.w};
                const uint32_t nv[4] = {NV.x, NV.y, NV.z, NV.w};
                if (4 * g + 4 > n)                             // slots past n hold no atom
#pragma unroll
                    for (int u = 1; u < 4; ++u)
                        if (4 * g + u >= n) x[u] = 0u;
                if ((x[0] | x[1] | x[2] | x[3]) != 0u) {
                    bool moved = false;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (x[u] == 0u) continue;
                        uint32_t xm = 0u;
                        const int el = tp_move(x[u], vx[u], d.tp_scale, &xm);
                        if (el >= 0) {                          // sticks at an electrode
                            tp_stick(d, B, 4 * g + u, el, vx[u]);
                            x[u] = 0u;
                            continue;
                        }
                        x[u] = xm;
                        if (nv[u] == 0u || (int)(nv[u] - 1u - s) <= 0) {   // a candidate due, or no gap yet
                            bool hit;
                            vx[u] = tp_candidate<LAW>(d, B, 4 * g + u, s, vx[u], nv[u], &hit);
                            if (hit) {
                                moved = true;
                                ++ncoll;
                            }
                        }
                        if (sample) {
                            uint32_t j, wr;
                            cell_of(x[u], d.kshift, j, wr);
                            if (j != run.j) {
                                tp_run_flush(A, run);
                                run.j = j;
                            }
                            const long long vq = (long long)__float2int_rn(vx[u]);
                            const long long w16 = (long long)(wr >> 16);
                            run.cnt += 1u;
                            run.whi += wr >> 16;
                            run.wlo += wr & 0xffffu;
                            run.f0 += vq * (65536 - w16);
                            run.f1 += vq * w16;
                        }
                    }
                    ((uint4*)B.pos)[g] = make_uint4(x[0], x[1], x[2], x[3]);
                    if (moved) ((float4*)B.vx)[g] = make_float4(vx[0], vx[1], vx[2], vx[3]);
                }
            }
            __syncwarp();                                     // the stage is read: refill it
            tile[st] = claim(st);
        }
        if (sample) {                                          // this span's tallies into the step's histograms
            tp_run_flush(A, run);
            run.j = kTpNoRun;
            __syncthreads();
            tp_flush(A, N, d.tp_q, d.tp_flux, threadIdx.x, blockDim.x);
            if (threadIdx.x == 0) s_tile = 0;
            __syncthreads();
        }
    }
    ncoll = __reduce_add_sync(0xffffffffu, ncoll);
    if (lane == 0 && ncoll) atomicAdd(&s_coll, ncoll);
    __syncthreads();
    if (threadIdx.x == 0 && s_coll) atomicAdd(&ctl->cnt[kCntTpColl], (unsigned long long)s_coll);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ctl->tp_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int m = threadIdx.x; m <= N; m += blockDim.x) {
        if (sample) {
            red_split(d.diag.tp_dens + 2 * m, __ldcg(d.tp_q + m));
            red_split_signed(d.diag.tp_vx + 2 * m, __ldcg(d.tp_flux + m));
        }
        d.tp_q[m] = 0;
        d.tp_flux[m] = 0;
    }
    if (threadIdx.x == 0) {
        ctl->tp_step = s + 1;
        if (sample) ctl->n_tp_samp += 1;
        ctl->tp_done = 0;
    }
}

// ---------------------------------------------------------------- event-driven flight
// The gridless alternative to the per-step collision test (Sec. "Kinetic
// Particle Simulation": free flight tau = -tau_c ln R_f between events; Sec.
// "Limitations and Constraints": densities weighted by flight duration).  For
// hard spheres in a Maxwellian gas the rate is nu(v) = n sigma <|v - w|>, the
// relative speed averaged over the gas; at a collision the partner has the
// density |v - w| f(w) / <|v - w|>, drawn by rejection from the proposal
// (|v| + |w|) f(w): with probability |v| / (|v| + <|w|>) a Maxwellian w,
// otherwise a Maxwellian weighted by |w| (|w|^2 / c^2 = -ln(R1 R2), direction
// isotropic), accepted with probability |v - w| / (|v| + |w|).  Event e of an
// atom draws Philox(id, e, TPF_FLIGHT), (id, e, TPF_PARTNER + 2t [+1]) for
// proposal t and (id, e, TPF_SCATTER); e is kept per atom (SpBuf::nev).  One
// thread takes one atom through up to kmax events per launch.
constexpr int kTpfTries = 64;                     // proposals per collision (each accepted w.p. >= 1/2)

__device__ __forceinline__ float mean_rel_speed(float vm, float c)
{
    const float s = vm / c;
    if (s < 1e-3f) return 1.1283792f * c * (1.0f + s * s * (1.0f / 3.0f));
    return c * ((s + 0.5f / s) * erff(s) + expf(-s * s) * 0.5641896f);
}

// Per-CTA tallies of a flight launch in shared memory, flushed once per
// CTA: each cell array (residence time and path, partial-cell terms and
// difference arrays) as two 32-bit parts, value = hi 2^16 + lo with lo = the
// low 16 bits, and the Al deposition histograms.  A CTA takes at most
// kTpfAtomsPerCta atoms through at most kTpfMaxEvents events, so a part sums
// at most 1024 x 33 values below 2^16 (lo) or 2^14 (hi) and cannot
// overflow; a value of 2^30 or more goes to global memory directly.
constexpr int kTpfAtomsPerCta = 1024;
constexpr int kTpfMaxEvents = 32;
struct TpfAcc {
    unsigned int* lo;         // [4][N+1]: tpart, tdiff, dpart, ddiff
    int* hi;                  // [4][N+1]
    unsigned int* spe;        // [2][kNbSpE]
    unsigned int* spa;        // [2][kNbAng]
    int n1;                   // N + 1
};

size_t tpf_smem(int N) { return (size_t)8 * 4 * (N + 1) + (size_t)4 * 2 * (kNbSpE + kNbAng); }

__device__ __forceinline__ void tpf_add(const TpfAcc& A, long long* g, int k, int i, long long v)
{
    if (!v) return;
    if (v >= (1ll << 30) || v <= -(1ll << 30)) {
        atomicAdd((unsigned long long*)&g[i], (unsigned long long)v);
        return;
    }
    atomicAdd(&A.lo[k * A.n1 + i], (unsigned int)(v & 0xffff));
    const int h = (int)(v >> 16);
    if (h) atomicAdd(&A.hi[k * A.n1 + i], h);
}

// residence time and signed path of the straight segment x0 -> x1 (fixed
// point) flown at v_x; tau only where v_x = 0 (the atom stays in its cell)
__device__ void tpf_segment(const Dev& d, const TpfAcc& A, long long x0, long long x1, float vx, float tau)
{
    const int S = 32 - d.kshift, N = d.ncell;
    const Diag& g = d.diag;
    if (vx == 0.0f || x0 == x1) {
        const int j = min(N - 1, (int)(x0 >> S));
        tpf_add(A, g.tpf_tpart, 0, j, __float2ll_rn(tau * 1099511627776.0f));
        return;
    }
    const long long lo = min(x0, x1), hi = max(x0, x1);
    const long long sg = vx > 0.0f ? 1 : -1;
    const float kt = d.tpf_kt / fabsf(vx);        // 2^-40 s per fixed-point unit
    const int ja = min(N - 1, (int)(lo >> S)), jb = min(N - 1, (int)((hi - 1) >> S));
    if (ja == jb) {
        tpf_add(A, g.tpf_tpart, 0, ja, __float2ll_rn((float)(hi - lo) * kt));
        tpf_add(A, g.tpf_dpart, 2, ja, sg * (hi - lo));
        return;
    }
    const long long oa = ((long long)(ja + 1) << S) - lo, ob = hi - ((long long)jb << S);
    tpf_add(A, g.tpf_tpart, 0, ja, __float2ll_rn((float)oa * kt));
    tpf_add(A, g.tpf_tpart, 0, jb, __float2ll_rn((float)ob * kt));
    tpf_add(A, g.tpf_dpart, 2, ja, sg * oa);
    tpf_add(A, g.tpf_dpart, 2, jb, sg * ob);
    if (jb > ja + 1) {                            // the cells crossed whole
        const long long tc = __float2ll_rn((float)(1ll << S) * kt);
        tpf_add(A, g.tpf_tdiff, 1, ja + 1, tc);
        tpf_add(A, g.tpf_tdiff, 1, jb, -tc);
        tpf_add(A, g.tpf_ddiff, 3, ja + 1, sg << S);
        tpf_add(A, g.tpf_ddiff, 3, jb, -(sg << S));
    }
}

// kmax <= kTpfMaxEvents; CTA b takes atoms [b kTpfAtomsPerCta, (b + 1) kTpfAtomsPerCta)
template <bool LAW>
__global__ void __launch_bounds__(kTpThreads) k_tp_flight(Dev d, int kmax)
{
    extern __shared__ __align__(16) unsigned char tpf_raw[];
    Ctl* ctl = d.ctl;
    const int N1 = d.ncell + 1;
    TpfAcc A;
    A.n1 = N1;
    A.lo = (unsigned int*)tpf_raw;
    A.hi = (int*)tpf_raw + (size_t)4 * N1;
    A.spe = (unsigned int*)tpf_raw + (size_t)8 * N1;
    A.spa = A.spe + 2 * kNbSpE;
    __shared__ unsigned int s_cnt[4];             // alive, collisions, deposited left, right
    __shared__ unsigned int s_next;               // next atom of the CTA's range to take
    for (int i = threadIdx.x; i < 8 * N1 + 2 * (kNbSpE + kNbAng); i += blockDim.x) ((unsigned int*)tpf_raw)[i] = 0;
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0;
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();

    const SpBuf B = d.buf[kTP][ctl->cur[kTP]];
    const long long n = ctl->n[kTP];
    const float c = d.tpf_c, vg = 0.70710678f * d.tpf_c, mw = 1.1283792f * d.tpf_c;
    const float mu_al = (float)(kMAL / (kMAL + kMAR)), mu_ar = (float)(kMAR / (kMAL + kMAR));
    const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
    unsigned int n_alive = 0, n_coll = 0, n_dep_l = 0, n_dep_r = 0;
    const long long a0 = (long long)blockIdx.x * kTpfAtomsPerCta;
    const long long na = min(n, a0 + kTpfAtomsPerCta) - a0;
    // each thread takes the CTA's atoms one after another from a shared
    // counter and runs one event per loop iteration, so the lanes of a warp
    // stay on the same code whatever the number of events of their atoms
    long long k = -1;
    uint32_t x = 0u, e = 0u;
    uint64_t id = 0;
    float vx = 0.0f, vy = 0.0f, vz = 0.0f;
    int ev = 0;
    for (;;) {
        if (k < 0) {                                               // take the next live atom
            const long long q = (long long)atomicAdd(&s_next, 1u);
            if (q >= na) break;
            const long long kk = a0 + q;
            x = ((const uint32_t*)B.pos)[kk];
            if (x == 0u) continue;
            k = kk;
            vx = B.vx[k]; vy = B.vy[k]; vz = B.vz[k];
            id = B.id[k];
            e = B.nev[k];
            ev = 0;
        }
        bool done = false, live = true;
        const float vm = sqrtf(vx * vx + vy * vy + vz * vz);
        // hard spheres: the exact rate; VHS / M1: the majorant n K (|v|^alpha + <|w|^alpha>)
        const float va = LAW ? powf(vm, d.tp_alpha) : 0.0f;
        const float nu = LAW ? d.tpf_nK * (va + d.tpf_malpha) : d.tpf_nsig * mean_rel_speed(vm, c);
        const uint4 f = draw(d.seed, id, e, kPurTpfFlight);
        const float tau = nu > 0.0f ? -logf(u23(f.x)) / nu : INFINITY;
        if (!(tau < INFINITY) && vx == 0.0f) {
            done = true;                                           // no gas, no motion across the gap
        } else {
            const float disp = vx * tau * d.tpf_scale;
            long long x1 = 0;
            int el = -1;
            if (!(fabsf(disp) < 8.0e9f)) {
                el = disp < 0.0f ? 0 : 1;
            } else {
                x1 = (long long)x + __float2ll_rn(disp);
                if (x1 <= 0) el = 0;
                else if (x1 >= 4294967296LL) el = 1;
            }
            if (el >= 0) {                                         // sticks at an electrode
                tpf_segment(d, A, x, el == 0 ? 0ll : 4294967296LL, vx, tau);
                const float E = vm * vm * (float)(0.5 * kMAL / kQE);
                const float ct = fminf(vm > 0.0f ? fabsf(vx) / vm : 1.0f, 1.0f);
                const int be = hist_bin(E, 300.0f, kNbSpE);
                const int ba = clamp_bin(acosf(ct) * (float)(180.0 / kPI), kNbAng);
                atomicAdd(&A.spe[el * kNbSpE + be], 1u);
                atomicAdd(&A.spa[el * kNbAng + ba], 1u);
                if (el == 0) ++n_dep_l;
                else ++n_dep_r;
                live = false;
                done = true;
            } else {
                tpf_segment(d, A, x, x1, vx, tau);
                x = (uint32_t)x1;
                // the collision partner, flux-weighted (hard spheres), or a candidate
                // partner and the test whether it is a real collision (VHS / M1)
                float wx = 0.0f, wy = 0.0f, wz = 0.0f, gm = 0.0f;
                bool real = true;
                for (int t = 0; !LAW && t < kTpfTries; ++t) {
                    uint4 cw[2];
                    cw[0] = make_uint4((uint32_t)id, (uint32_t)(id >> 32), e, kPurTpfPartner + 2 * t);
                    cw[1] = make_uint4((uint32_t)id, (uint32_t)(id >> 32), e, kPurTpfPartner + 2 * t + 1);
                    philox_n<2>(cw, k0, k1);
                    const uint4 a = cw[0], b = cw[1];
                    if (u23(a.x) * (vm + mw) < vm) {
                        const float2 n12 = box_muller(a.y, a.z), n34 = box_muller(a.w, b.x);
                        wx = vg * n12.x; wy = vg * n12.y; wz = vg * n34.x;
                    } else {
                        const float sp = c * sqrtf(-logf(u23(a.y) * u23(a.z)));
                        const float3 dd = iso_dir(a.w, b.x);
                        wx = sp * dd.x; wy = sp * dd.y; wz = sp * dd.z;
                    }
                    const float gx = vx - wx, gy = vy - wy, gz = vz - wz;
                    gm = sqrtf(gx * gx + gy * gy + gz * gz);
                    const float wm = sqrtf(wx * wx + wy * wy + wz * wz);
                    if (u23(b.y) * (vm + wm) < gm) break;
                }
                if (LAW) {
                    uint4 cw[2];
                    cw[0] = make_uint4((uint32_t)id, (uint32_t)(id >> 32), e, kPurTpfCand);
                    cw[1] = make_uint4((uint32_t)id, (uint32_t)(id >> 32), e, kPurTpfCand + 1);
                    philox_n<2>(cw, k0, k1);
                    const uint4 a = cw[0], b = cw[1];
                    if (u23(a.x) * (va + d.tpf_malpha) < va) {
                        const float2 n12 = box_muller(a.y, a.z), n34 = box_muller(a.w, b.x);
                        wx = vg * n12.x; wy = vg * n12.y; wz = vg * n34.x;
                    } else {
                        const float sp = c * sqrtf(gamma_mt(d.tpf_gk, d.seed, id, e, kPurTpfGamma));
                        const float3 dd = iso_dir(a.w, b.x);
                        wx = sp * dd.x; wy = sp * dd.y; wz = sp * dd.z;
                    }
                    const float gx = vx - wx, gy = vy - wy, gz = vz - wz;
                    gm = sqrtf(gx * gx + gy * gy + gz * gz);
                    const float wm = sqrtf(wx * wx + wy * wy + wz * wz);
                    real = u23(b.y) * (va + powf(wm, d.tp_alpha)) < powf(gm, d.tp_alpha);
                }
                if (real) {                                        // scattering in the centre of mass
                    const uint4 sc = draw(d.seed, id, e, kPurTpfScatter);
                    const float3 dir = LAW ? tp_scatter_dir(d.tp_model, vx - wx, vy - wy, vz - wz, gm, sc.x, sc.y)
                                           : iso_dir(sc.x, sc.y);
                    vx = mu_al * vx + mu_ar * wx + mu_ar * gm * dir.x;
                    vy = mu_al * vy + mu_ar * wy + mu_ar * gm * dir.y;
                    vz = mu_al * vz + mu_ar * wz + mu_ar * gm * dir.z;
                    ++n_coll;
                }
                ++e;
                done = ++ev == kmax;
            }
        }
        if (done) {                                                // the atom leaves this launch
            ((uint32_t*)B.pos)[k] = live ? x : 0u;
            B.vx[k] = vx;
            B.vy[k] = vy;
            B.vz[k] = vz;
            B.nev[k] = e;
            n_alive += live ? 1u : 0u;
            k = -1;
        }
    }
    const unsigned int cnt[4] = {n_alive, n_coll, n_dep_l, n_dep_r};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const unsigned int v = __reduce_add_sync(0xffffffffu, cnt[i]);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_cnt[i], v);
    }
    __syncthreads();
    const Diag& g = d.diag;
    for (int i = threadIdx.x; i < 4 * N1; i += blockDim.x) {
        const int k = i / N1, m = i - k * N1;
        long long* dst = k == 0 ? g.tpf_tpart : (k == 1 ? g.tpf_tdiff : (k == 2 ? g.tpf_dpart : g.tpf_ddiff));
        const long long v = ((long long)A.hi[i] << 16) + (long long)A.lo[i];
        if (v) atomicAdd((unsigned long long*)&dst[m], (unsigned long long)v);
    }
    for (int i = threadIdx.x; i < 2 * kNbSpE; i += blockDim.x)
        if (A.spe[i]) atomicAdd(&g.sp_e[i / kNbSpE][i % kNbSpE], (unsigned long long)A.spe[i]);
    for (int i = threadIdx.x; i < 2 * kNbAng; i += blockDim.x)
        if (A.spa[i]) atomicAdd(&g.sp_ang[i / kNbAng][i % kNbAng], (unsigned long long)A.spa[i]);
    if (threadIdx.x == 0) {
        if (s_cnt[0]) atomicAdd(&ctl->tpf_alive, (unsigned long long)s_cnt[0]);
        if (s_cnt[1]) atomicAdd(&ctl->cnt[kCntTpColl], (unsigned long long)s_cnt[1]);
        if (s_cnt[2]) atomicAdd(&ctl->cnt[kCntTpDepL], (unsigned long long)s_cnt[2]);
        if (s_cnt[3]) atomicAdd(&ctl->cnt[kCntTpDepR], (unsigned long long)s_cnt[3]);
    }
}

// Mono-energetic ion source on the left electrode: n atoms with Thompson
// energies (cut off at Lambda E_ion) and cosine angles, ids tag | (id0 + k).
__global__ void k_tp_launch(Dev d, long long n, long long id0, float Emax)
{
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long base = d.ctl->n[kTP];
    const long long idx = base + k;
    const uint64_t id = id_tag(kTP) | (uint64_t)(id0 + k);
    if (idx >= d.ctl->cap[kTP]) {
        atomicOr(&d.ctl->err, kErrCapacity);
        return;
    }
    const SpBuf B = d.buf[kTP][d.ctl->cur[kTP]];
    const uint4 ce = draw(d.seed, id, 0, kPurTpLaunch);
    const float3 v = emit(u23(ce.x), u23(ce.y), u23(ce.z), Emax, 1.0f);
    ((uint32_t*)B.pos)[idx] = 1u;
    B.vx[idx] = v.x;
    B.vy[idx] = v.y;
    B.vz[idx] = v.z;
    B.id[idx] = id;
    B.nev[idx] = 0u;
}

__global__ void k_commit_count(Dev d, int s, long long add)
{
    long long n = d.ctl->n[s] + add;
    d.ctl->n[s] = n > d.ctl->cap[s] ? d.ctl->cap[s] : n;
}

size_t tp_smem(int ncell) { return (size_t)ncell * 12 + (size_t)(ncell + 1) * 8; }

cudaError_t launch_tp_flight(const Dev& d, int kmax, long long n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (kmax > kTpfMaxEvents) kmax = kTpfMaxEvents;
    const size_t sm = tpf_smem(d.ncell);
    if (sm > 48 * 1024) {
        const void* fn = d.tp_model ? (const void*)k_tp_flight<true> : (const void*)k_tp_flight<false>;
        const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    const long long grid = (n + kTpfAtomsPerCta - 1) / kTpfAtomsPerCta;
    if (d.tp_model) k_tp_flight<true><<<(unsigned)grid, kTpThreads, sm, st>>>(d, kmax);
    else k_tp_flight<false><<<(unsigned)grid, kTpThreads, sm, st>>>(d, kmax);
    return cudaGetLastError();
}

static const void* tp_step_fn(const Dev& d, bool sample)
{
    if (d.tp_mode != 0) return d.tp_model ? (const void*)k_tp_step<true> : (const void*)k_tp_step<false>;
    if (sample) return d.tp_model ? (const void*)k_tp_step_geo<true, true> : (const void*)k_tp_step_geo<false, true>;
    return d.tp_model ? (const void*)k_tp_step_geo<true, false> : (const void*)k_tp_step_geo<false, false>;
}

static size_t tp_step_smem(const Dev& d, bool sample)
{
    return d.tp_mode == 0 ? (sample ? tp_geo_smem(d.ncell) : tp_ring_smem(d.ncell)) : tp_smem(d.ncell);
}

cudaError_t tp_occupancy(const Dev& d, bool sample, int* blocks_per_sm)
{
    const size_t sm = tp_step_smem(d, sample);
    if (sm > 40 * 1024) {                  // (with the static shared memory, 48 KB of rings pass the default limit)
        const cudaError_t e = cudaFuncSetAttribute(tp_step_fn(d, sample), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, tp_step_fn(d, sample), kTpThreads, sm);
}

cudaError_t launch_tp_step(const Dev& d, int grid, bool sample, cudaStream_t st)
{
    const size_t sm = tp_step_smem(d, sample);
    const void* fn = tp_step_fn(d, sample);
    if (sm > 40 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    if (d.tp_mode == 0) {
        if (sample) {
            if (d.tp_model) k_tp_step_geo<true, true><<<grid, kTpThreads, sm, st>>>(d);
            else k_tp_step_geo<false, true><<<grid, kTpThreads, sm, st>>>(d);
        } else {
            if (d.tp_model) k_tp_step_geo<true, false><<<grid, kTpThreads, sm, st>>>(d);
            else k_tp_step_geo<false, false><<<grid, kTpThreads, sm, st>>>(d);
        }
    } else {
        if (d.tp_model) k_tp_step<true><<<grid, kTpThreads, sm, st>>>(d);
        else k_tp_step<false><<<grid, kTpThreads, sm, st>>>(d);
    }
    return cudaGetLastError();
}

cudaError_t launch_tp_launch(const Dev& d, long long n, long long id0, float Emax, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int T = 256;
    k_tp_launch<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(d, n, id0, Emax);
    k_commit_count<<<1, 1, 0, st>>>(d, kTP, n);
    return cudaGetLastError();
}

}  // namespace pg
