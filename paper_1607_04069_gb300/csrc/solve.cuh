// solve.cuh -- one-CTA field solve for the 1D electrostatic PIC cycle.
//
// Poisson's equation discretised as in the paper's field-solver paragraph
// (Sec. "EM Field Solver and External Lumped Circuits"):
//     (phi[m+1] - 2 phi[m] + phi[m-1]) / dx^2 = -rho[m] / eps0,  m = 1..N-1,
// with phi[0] = V_rf(t), phi[N] = 0, and E[m] = -(phi[m+1] - phi[m-1]) / (2 dx).
// With rho[m] = e w q[m] / (2^32 dx) (q in units of 2^-32 superparticles)
// the rows read  phi[m+1] - 2 phi[m] + phi[m-1] = -A q[m],
// A = dx e w / (2^32 eps0).  For this constant-coefficient Dirichlet system
// the Thomas elimination collapses to two prefix sums:
//     S_m = sum_{j=1..m} q[j],   T_m = sum_{k<m} S_k,
//     D0  = (phi[N] - phi[0] + A T_N) / N,
//     phi[m] = phi[0] + m D0 - A T_m,
//     E[m]   = -(2 D0 - A (S_m + S_{m-1})) / (2 dx)              (inside),
//     E[0]   = -(D0 + A q[0]) / dx,   E[N] = -(D0 - A S_N) / dx  (half-cell Gauss).
// S is summed in int64 and T in int128, so both are exact and independent of
// the block shape; the only roundings are the final FP64 products.
#pragma once
#include "common.cuh"

namespace pg {

__device__ __forceinline__ long long shfl_up_t(long long v, int d)
{
    return __shfl_up_sync(0xffffffffu, v, d);
}
__device__ __forceinline__ __int128 shfl_up_t(__int128 v, int d)
{
    const unsigned long long lo = (unsigned long long)v;
    const long long hi = (long long)(v >> 64);
    const unsigned long long lo2 = __shfl_up_sync(0xffffffffu, lo, d);
    const long long hi2 = __shfl_up_sync(0xffffffffu, hi, d);
    return (__int128)(((unsigned __int128)(unsigned long long)hi2 << 64) | lo2);
}

// Exclusive scan over the block (blockDim.x a multiple of 32, <= 1024).
// `sh` must hold 32 elements.  `total` receives the block total.
template <typename T>
__device__ T block_exclusive_scan(T v, T* sh, T& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T y = shfl_up_t(x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T w = lane < nw ? sh[lane] : (T)0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const T y = shfl_up_t(w, d);
            if (lane >= d) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    const T off = wid ? sh[wid - 1] : (T)0;
    total = sh[nw - 1];
    __syncthreads();
    return off + x - v;
}

__device__ __forceinline__ double i128_to_double(__int128 x)
{
    const bool neg = x < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)(-x) : (unsigned __int128)x;
    const double d = (double)(unsigned long long)(u >> 64) * 18446744073709551616.0 +
                     (double)(unsigned long long)u;
    return neg ? -d : d;
}

// net charge count at node m: ions minus electrons
struct QNet {
    const unsigned long long* qi;
    const unsigned long long* qe;
    bool cg;   // read through L2 (data written by atomics of other CTAs of this kernel)
    __device__ __forceinline__ long long operator()(int m) const
    {
        const unsigned long long a = cg ? __ldcg(qi + m) : qi[m];
        const unsigned long long b = cg ? __ldcg(qe + m) : qe[m];
        return (long long)(a - b);
    }
};

// Series blocking capacitor, for the solves below: with circ non-null the
// electrode potential is not v_left but follows from the source voltage
// v_left, the deposit and the charge absorbed at x = 0 (Dev::circ_a).
struct CircuitArgs {
    double a, b;          // Dev::circ_a, Dev::circ_b
    long long dn;         // Ctl::wall_dn
};

// Solve for phi and E with one CTA.  Any output pointer may be null.
// Returns the electrode potential phi[0].
__device__ __noinline__ static double poisson_block(const QNet& qn, int N, double A, double inv_dx, double v_left,
                                                    double* phi, double* E64, float* E32,
                                                    const CircuitArgs* circ = nullptr)
{
    __shared__ long long sh64[32];
    __shared__ __int128 sh128[32];
    const int T = blockDim.x, t = threadIdx.x;
    const int N1 = N + 1;
    const int seg = (N1 + T - 1) / T;
    const int m0 = min(t * seg, N1), m1 = min(m0 + seg, N1);

    long long a = 0;
    for (int m = m0; m < m1; ++m)
        if (m >= 1) a += qn(m);
    long long totS;
    const long long Sprev = block_exclusive_scan(a, sh64, totS);

    __int128 b = 0;
    long long S = Sprev;
    for (int m = m0; m < m1; ++m) {
        if (m >= 1) S += qn(m);
        b += (__int128)S;
    }
    __int128 totT;
    const __int128 Tpre = block_exclusive_scan(b, sh128, totT);
    const __int128 TN = totT - (__int128)totS;
    if (circ) {
        const __int128 X = TN + (__int128)N * (__int128)qn(0) + ((__int128)N << 32) * (__int128)circ->dn;
        v_left = 0.5 * A * (circ->a * v_left + circ->b * i128_to_double(X));
    }
    const double D0 = (0.0 - v_left + A * i128_to_double(TN)) / (double)N;

    S = Sprev;
    __int128 Tm = Tpre;
    for (int m = m0; m < m1; ++m) {
        const long long q = qn(m);
        const long long Sm = m >= 1 ? S + q : 0;
        const double ph = v_left + (double)m * D0 - A * i128_to_double(Tm);
        double E;
        if (m == 0) E = -(D0 + A * (double)q) * inv_dx;
        else if (m == N) E = -(D0 - A * (double)Sm) * inv_dx;
        else E = -(2.0 * D0 - A * (double)(Sm + S)) * (0.5 * inv_dx);
        if (phi) phi[m] = ph;
        if (E64) E64[m] = E;
        if (E32) E32[m] = (float)E;
        Tm += (__int128)Sm;
        S = Sm;
    }
    return v_left;
}

// Field at the nodes in FP32 from the exact integer sums, for the gather of
// one CTA.  With S_m as above and K an integer close to 2 D0 / A,
//     E[m] = c1 + c2 (S_m + S_{m-1} - K),  c2 = A / (2 dx),  c1 = -D0/dx + c2 K,
//     E[0] = c1 + c2 (-K - 2 q[0]),        E[N] = c1 + c2 (2 S_N - K),
// which is the central difference and the half-cell Gauss rule above: the
// bracket is an exact int64, so each E[m] is one rounding of its own value.
// K and c1 follow from T_N = sum_{j=1}^{N-1} (N - j) q_j in integer
// arithmetic: with 2 V / A = va_i + va_f,
//     2 D0 / A = (2 T_N - va_i - va_f) / N,  K = round((2 T_N - va_i) / N),
//     c1 = c2 (va_f - rem) / N,  rem = 2 T_N - va_i - K N,
// so no FP64 arithmetic runs per step (N is a power of two).  All warps of
// the CTA take part; one block barrier.  qe, qi: shared copies of the
// deposit; sE: shared float[N+1].
// Returns the electrode potential phi[0] of the solve; with the series
// capacitor (field_mode kFieldCircuit) it is formed here from the source
// voltage a.v_left, T_N, q_0 and the charge absorbed at x = 0, as 2 phi_0/A =
// circ_a V + circ_b (T_N + N q_0 + N 2^32 dn), and then split as above.
// wall_dn: Ctl::wall_dn, loaded by the caller at the start of the launch.
__device__ static double block_field_f32(const Dev& d, const unsigned long long* qe, const unsigned long long* qi,
                                         float* sE, const StepArgs& a, long long wall_dn)
{
    __shared__ long long s_wacc[32], s_wbhi[32];
    __shared__ unsigned long long s_wblo[32];
    const unsigned FULL = 0xffffffffu;
    const int N = d.ncell, N1 = N + 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (a.field_mode == kFieldUniform) {
        for (int m = threadIdx.x; m < N1; m += blockDim.x) sE[m] = a.e_uniform;
        return a.v_left;
    }
    // nodes of this warp, then of this lane
    const int w0 = N1 * w / nw, w1 = N1 * (w + 1) / nw;
    const int seg = (w1 - w0 + 31) / 32;
    const int m0 = min(w0 + lane * seg, w1), m1 = min(m0 + seg, w1);
    long long acc = 0, bhi = 0;
    unsigned long long blo = 0;
    for (int m = m0; m < m1; ++m) {
        if (m < 1) continue;
        const long long q = (long long)(qi[m] - qe[m]);
        const unsigned int wt = (unsigned int)(N - m);
        acc += q;
        blo += (unsigned long long)(unsigned int)q * wt;     // (N - m) q = (q_hi 2^32 + q_lo)(N - m)
        bhi += (q >> 32) * (long long)wt;
    }
    long long incl = acc;
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
        const long long y = __shfl_up_sync(FULL, incl, k);
        if (lane >= k) incl += y;
    }
    unsigned long long rlo = blo;
    long long rhi = bhi;
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) {
        rlo += __shfl_xor_sync(FULL, rlo, k);
        rhi += __shfl_xor_sync(FULL, rhi, k);
    }
    if (lane == 31) s_wacc[w] = incl;
    if (lane == 0) {
        s_wblo[w] = rlo;
        s_wbhi[w] = rhi;
    }
    __syncthreads();
    long long Sw = 0;
    __int128 TN = 0;
    for (int k = 0; k < nw; ++k) {
        if (k < w) Sw += s_wacc[k];
        TN += ((__int128)s_wbhi[k] << 32) + (__int128)s_wblo[k];
    }
    long long K;
    float c1;
    const float c2 = d.c2f;
    int mode = a.field_mode;
    long long va_i = a.va_i;
    float va_f = a.va_f;
    double v_el = a.v_left;
    if (mode == kFieldCircuit) {
        const long long q0 = (long long)(qi[0] - qe[0]);
        const __int128 X = TN + (__int128)N * q0 + ((__int128)N << 32) * (__int128)wall_dn;
        const double va = d.circ_a * a.v_left + d.circ_b * i128_to_double(X);
        v_el = 0.5 * d.A * va;
        if (fabs(va) < 4.0e18) {
            va_i = llrint(va);
            va_f = (float)(va - (double)va_i);
            mode = kFieldInt;
        } else {
            mode = kFieldF64;
        }
    }
    if (mode == kFieldInt) {
        const __int128 x = 2 * TN - (__int128)va_i;
        const __int128 Kq = (x + (__int128)(N >> 1)) >> d.kshift;
        const long long rem = (long long)(x - (Kq << d.kshift));
        K = (long long)Kq;
        c1 = c2 * ((va_f - (float)rem) / (float)N);
    } else {
        const double D0 = (0.0 - v_el + d.A * i128_to_double(TN)) / (double)N;
        const double k = 2.0 * D0 / d.A;
        K = fabs(k) < 4e18 ? llrint(k) : 0;
        c1 = (float)(-D0 * d.inv_dx + 0.5 * d.A * d.inv_dx * (double)K);
    }
    long long S = Sw + incl - acc;                     // S_{m0 - 1}
    for (int m = m0; m < m1; ++m) {
        const long long q = (long long)(qi[m] - qe[m]);
        const long long Sm = m >= 1 ? S + q : 0;
        long long br;
        if (m == 0) br = -K - 2 * q;
        else if (m == N) br = 2 * Sm - K;
        else br = Sm + S - K;
        sE[m] = c1 + c2 * (float)br;
        S = Sm;
    }
    return v_el;
}

// Add the state of step l (deposit in slot l%3; the flux moment sampled at
// step l) to the time averages for nodes [m0, m1); `count`: this CTA also
// counts the step (exactly one CTA per step does).
__device__ static void accumulate_nodes(const Dev& d, unsigned int l, const unsigned long long* qe,
                                        const unsigned long long* qi, int m0, int m1, double v_left,
                                        bool count, int t, int nt)
{
    const bool fl = d.diag_every > 0 && l > 0 && l % (unsigned)d.diag_every == 0;
    const int slot = l % 3;
    for (int m = m0 + t; m < m1; m += nt) {
        red_split(d.diag.sum_q[kE] + 2 * m, qe[m]);
        red_split(d.diag.sum_q[kI] + 2 * m, qi[m]);
        if (fl) {
            red_split_signed(d.diag.sum_flux[kE] + 2 * m, d.fbuf[slot][kE][m]);
            red_split_signed(d.diag.sum_flux[kI] + 2 * m, d.fbuf[slot][kI][m]);
        }
    }
    if (count && t == 0) {
        Ctl* c = d.ctl;
        c->sum_v += v_left;
        c->n_avg += 1;
        if (fl) c->n_flux += 1;
    }
}

// Bookkeeping at the end of a launch, by its last CTA: advance the step and
// take the births of this launch into the slot counts.
__device__ static void commit_step(const Dev& d, bool advance)
{
    Ctl* c = d.ctl;
    if (advance) {
        c->step += 1;
        c->field_override = 0;
    }
    c->wall_dn += c->wall_delta;                  // every CTA of the launch has added its share
    c->wall_delta = 0;
    // charged-species births start at round_up(n, 4) (see k_mover), atoms at n
    for (int s = 0; s < 3; ++s) {
        if (c->births[s] == 0) continue;
        long long n = (s == kTP ? c->n[s] : ((c->n[s] + 3) & ~3ll)) + c->births[s];
        if (n > c->cap[s]) n = c->cap[s];
        c->n[s] = n;
        c->births[s] = 0;
    }
    c->done = 0;
}

}  // namespace pg
