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

__global__ void __launch_bounds__(kTpThreads) k_tp_step(Dev d)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N1 = d.ncell + 1;
    unsigned long long* sq = (unsigned long long*)smem_raw;
    long long* sflux = (long long*)(sq + N1);
    __shared__ unsigned int s_coll;
    __shared__ int s_last;

    Ctl* ctl = d.ctl;
    const unsigned int s = ctl->tp_step;
    const long long n = ctl->n[kTP];
    const bool sample = d.diag_every > 0 && ((s + 1) % (unsigned)d.diag_every == 0);
    const long long beg = n * blockIdx.x / gridDim.x, end = n * (blockIdx.x + 1) / gridDim.x;
    for (int i = threadIdx.x; i < N1; i += blockDim.x) {
        sq[i] = 0;
        sflux[i] = 0;
    }
    if (threadIdx.x == 0) s_coll = 0;
    __syncthreads();

    const SpBuf B = d.buf[kTP][ctl->cur[kTP]];
    uint32_t* __restrict__ P = (uint32_t*)B.pos;
    const float mu_al = (float)(kMAL / (kMAL + kMAR)), mu_ar = (float)(kMAR / (kMAL + kMAR));
    for (long long i0 = beg; i0 < end; i0 += blockDim.x) {
        const long long i = i0 + threadIdx.x;
        bool act = i < end;
        uint32_t x = 0;
        if (act) {
            x = P[i];
            act = x != 0u;
        }
        uint32_t j = 0, wr = 0;
        bool dep = false;
        if (act) {
            float vx = B.vx[i], vy = B.vy[i], vz = B.vz[i];
            const uint64_t id = B.id[i];
            const long long np = (long long)x + __float2ll_rn(vx * d.tp_scale);
            if (np <= 0 || np >= 4294967296LL) {
                const int el = np <= 0 ? 0 : 1;
                const float v2 = vx * vx + vy * vy + vz * vz;
                const float E = v2 * (float)(0.5 * kMAL / kQE);
                float ct = v2 > 0.0f ? fabsf(vx) * rsqrtf(v2) : 1.0f;
                ct = fminf(ct, 1.0f);
                int be = (int)(E / 300.0f * (float)kNbSpE);
                be = be < 0 ? 0 : (be > kNbSpE - 1 ? kNbSpE - 1 : be);
                int ba = (int)(acosf(ct) * (float)(180.0 / kPI));
                ba = ba < 0 ? 0 : (ba > kNbAng - 1 ? kNbAng - 1 : ba);
                atomicAdd(&d.diag.sp_e[el][be], 1ull);
                atomicAdd(&d.diag.sp_ang[el][ba], 1ull);
                atomicAdd(&ctl->cnt[el == 0 ? kCntTpDepL : kCntTpDepR], 1ull);
                P[i] = 0u;
            } else {
                x = (uint32_t)np;
                const uint4 cg = draw(d.seed, id, s, kPurTpGas);
                const float2 n12 = box_muller(cg.x, cg.y);
                const float2 n34 = box_muller(cg.z, cg.w);
                const float wx = d.vth_gas * n12.x, wy = d.vth_gas * n12.y, wz = d.vth_gas * n34.x;
                const float gx = vx - wx, gy = vy - wy, gz = vz - wz;
                const float gm = sqrtf(gx * gx + gy * gy + gz * gz);
                const float Pc = -expm1f(-d.tp_nsig_dt * gm);
                const uint4 cc = draw(d.seed, id, s, kPurTpColl);
                if (u23(cc.x) < Pc) {
                    const float3 dir = iso_dir(cc.y, cc.z);
                    vx = mu_al * vx + mu_ar * wx + mu_ar * gm * dir.x;
                    vy = mu_al * vy + mu_ar * wy + mu_ar * gm * dir.y;
                    vz = mu_al * vz + mu_ar * wz + mu_ar * gm * dir.z;
                    B.vx[i] = vx;
                    B.vy[i] = vy;
                    B.vz[i] = vz;
                    atomicAdd(&s_coll, 1u);
                }
                P[i] = x;
                if (sample) {
                    cell_of(x, d.kshift, j, wr);
                    dep = true;
                    const long long vq = (long long)__float2int_rn(vx);
                    atomicAdd((unsigned long long*)&sflux[j],
                              (unsigned long long)(vq * (long long)(((1ull << 32) - wr) >> 16)));
                    atomicAdd((unsigned long long*)&sflux[j + 1],
                              (unsigned long long)(vq * (long long)(wr >> 16)));
                }
            }
        }
        if (sample) warp_deposit(sq, dep, j, wr);
    }
    __syncthreads();
    if (sample) {
        for (int m = threadIdx.x; m < N1; m += blockDim.x) {
            if (sq[m]) atomicAdd(&d.tp_q[m], sq[m]);
            if (sflux[m]) atomicAdd((unsigned long long*)&d.tp_flux[m], (unsigned long long)sflux[m]);
        }
    }
    if (threadIdx.x == 0 && s_coll) atomicAdd(&ctl->cnt[kCntTpColl], (unsigned long long)s_coll);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ctl->tp_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int m = threadIdx.x; m < N1; m += blockDim.x) {
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
}

__global__ void k_commit_count(Dev d, int s, long long add)
{
    long long n = d.ctl->n[s] + add;
    d.ctl->n[s] = n > d.ctl->cap[s] ? d.ctl->cap[s] : n;
}

size_t tp_smem(int ncell) { return (size_t)(ncell + 1) * 16; }

cudaError_t launch_tp_step(const Dev& d, int grid, cudaStream_t st)
{
    const size_t sm = tp_smem(d.ncell);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute((const void*)k_tp_step,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_tp_step<<<grid, kTpThreads, sm, st>>>(d);
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
