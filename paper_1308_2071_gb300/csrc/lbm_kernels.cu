// Kernels of the single-cavity path: the fused collide-and-stream step, the
// observables pass, the final FP64 reductions with the Nusselt number, the
// state export, and the porosity conversion.
#include "lbm_internal.h"

namespace lbm {

// ---- fused step -------------------------------------------------------------------

// One time step for every node, pull form: each thread gathers the post-
// collision populations that stream into its node (Eq. 18, 35), applies the
// wall rule on perimeter nodes (Section 4), collides (Eq. 17, 34) and writes
// the node's post-collision populations to the other buffer.  The buffer
// pair alternates, so dst holds B_{n+1} when src holds B_n.
template <class S, class R, bool FIELD, class P>
__global__ void __launch_bounds__(256) k_step(const S* __restrict__ src, S* __restrict__ dst,
                                              const P* __restrict__ phi, Geom gm, Coef<R> c,
                                              int* __restrict__ status) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= gm.nx || y >= gm.ny) return;
    R d[9], h[5];
    Drag<R> dr;
    const Macro<R> mc = node_state<S, R, FIELD, P>(c, gm, src, phi, x, y, dr, d, h);
    if (!(mc.umag < R(0.5))) atomicOr(status, 1);  // also catches NaN
    collide<R>(c, dr.iphi, mc, d, h);
    const int off = y * gm.pitch + x;
#pragma unroll
    for (int i = 0; i < 9; ++i) Conv<S, R>::st(dst + i * gm.plane + off, d[i]);
#pragma unroll
    for (int j = 0; j < 5; ++j) Conv<S, R>::st(dst + (9 + j) * gm.plane + off, h[j]);
}

// ---- observables ------------------------------------------------------------------

// Block-wide reduction of four doubles: max, max, sum, sum.
__device__ __forceinline__ void block_reduce4(double v[4], double* sh /* 4 * 32 */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v[0] = fmax(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
        v[1] = fmax(v[1], __shfl_xor_sync(0xffffffffu, v[1], o));
        v[2] += __shfl_xor_sync(0xffffffffu, v[2], o);
        v[3] += __shfl_xor_sync(0xffffffffu, v[3], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) sh[k * 32 + warp] = v[k];
    }
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (lane < nw) ? sh[k * 32 + lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v[0] = fmax(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
            v[1] = fmax(v[1], __shfl_xor_sync(0xffffffffu, v[1], o));
            v[2] += __shfl_xor_sync(0xffffffffu, v[2], o);
            v[3] += __shfl_xor_sync(0xffffffffu, v[3], o);
        }
    }
}

// Macroscopic fields of the post-stream state S_n, rebuilt by pulling from
// B_{n-1} and applying the wall rule, plus per-block partials (FP64) of
// max|u|, max|u - u_prev|, sum of population deviations, sum of T - T0.
template <class S, class R, bool FIELD, class P>
__global__ void __launch_bounds__(256) k_observe(const S* __restrict__ prev, const P* __restrict__ phi,
                                                 Geom gm, Coef<R> c, R* ux_out, R* uy_out, R* T_out,
                                                 R* p_out, R* snap, int snap_valid,
                                                 double* __restrict__ partials) {
    __shared__ double sh[4 * 32];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const long n = (long)gm.nx * gm.ny;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const int y = (int)(k / gm.nx), x = (int)(k - (long)y * gm.nx);
        R d[9], h[5];
        Drag<R> dr;
        const Macro<R> mc = node_state<S, R, FIELD, P>(c, gm, prev, phi, x, y, dr, d, h);
        R sd = R(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) sd += d[i];
        if (ux_out) ux_out[k] = mc.ux;
        if (uy_out) uy_out[k] = mc.uy;
        if (T_out) T_out[k] = c.T0 + mc.dT;
        if (p_out) p_out[k] = (R(1.0 / 3.0) + mc.dP) * dr.iphi;
        double du = 0.0;
        if (snap) {
            if (snap_valid) {
                const double ax = (double)mc.ux - (double)snap[2 * k];
                const double ay = (double)mc.uy - (double)snap[2 * k + 1];
                du = sqrt(ax * ax + ay * ay);
            }
            snap[2 * k] = mc.ux;
            snap[2 * k + 1] = mc.uy;
        }
        v[0] = fmax(v[0], (double)mc.umag);
        v[1] = fmax(v[1], du);
        v[2] += (double)sd;
        v[3] += (double)mc.dT;
    }
    block_reduce4(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) partials[blockIdx.x * 4 + k] = v[k];
    }
}

// T - T0 of the post-stream state at node (x, y), pulled from B_{n-1}.
template <class S, class R>
__device__ __forceinline__ R node_dT(const Coef<R>& c, const Geom& gm, const S* __restrict__ prev,
                                     int x, int y) {
    const Normal nr = normal_of(gm, x, y);
    if (nr.dx == 0 && nr.dy == 0) return pull_heat<S, R>(prev, gm, y * gm.pitch + x) + c.qhalf;
    if (gm.thermal_bc == 1) return c.dTc;
    if (nr.dx != 0) return x == 0 ? c.dTh : c.dTc;
    const R dTf = pull_heat<S, R>(prev, gm, (y + nr.dy) * gm.pitch + x) + c.qhalf;
    if (gm.adi_order == 2) {
        const R dTff = pull_heat<S, R>(prev, gm, (y + 2 * nr.dy) * gm.pitch + x) + c.qhalf;
        return (R(4) * dTf - dTff) * R(1.0 / 3.0);
    }
    return dTf;
}

// One block: folds the per-block partials in a fixed order and evaluates the
// mean Nusselt numbers (Eq. 38) of both vertical walls, FP64 throughout:
// Nu(y) = -L dT/dx / dT with the one-sided five-point derivative
// (-25 T0 + 48 T1 - 36 T2 + 16 T3 - 3 T4) / 12, trapezoidal mean over y.
// out[0..6] = nu_hot, nu_cold, max|u|, max|du|, sum d, sum (T - T0), status.
template <class S, class R>
__global__ void __launch_bounds__(1024) k_finish(const S* __restrict__ prev, Geom gm, Coef<R> c,
                                                 const double* __restrict__ partials, int npart,
                                                 double L, double dT, const int* __restrict__ status,
                                                 double* __restrict__ out) {
    __shared__ double sh[4 * 32];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < npart; b += blockDim.x) {
        v[0] = fmax(v[0], partials[4 * b]);
        v[1] = fmax(v[1], partials[4 * b + 1]);
        v[2] += partials[4 * b + 2];
        v[3] += partials[4 * b + 3];
    }
    block_reduce4(v, sh);
    __syncthreads();
    double red[4] = {v[0], v[1], v[2], v[3]};
    __syncthreads();
    double w[4] = {0.0, 0.0, 0.0, 0.0};
    const int nx = gm.nx;
    for (int y = threadIdx.x; y < gm.ny; y += blockDim.x) {
        double tl[5], tr[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            tl[k] = (double)node_dT<S, R>(c, gm, prev, k, y);
            tr[k] = (double)node_dT<S, R>(c, gm, prev, nx - 1 - k, y);
        }
        const double dl = (-25.0 * tl[0] + 48.0 * tl[1] - 36.0 * tl[2] + 16.0 * tl[3] - 3.0 * tl[4]) / 12.0;
        const double dr = (25.0 * tr[0] - 48.0 * tr[1] + 36.0 * tr[2] - 16.0 * tr[3] + 3.0 * tr[4]) / 12.0;
        const double wt = (y == 0 || y == gm.ny - 1) ? 0.5 : 1.0;
        w[2] += wt * (-L * dl / dT);
        w[3] += wt * (-L * dr / dT);
    }
    block_reduce4(w, sh);
    if (threadIdx.x == 0) {
        out[0] = w[2] / (double)(gm.ny - 1);
        out[1] = w[3] / (double)(gm.ny - 1);
        out[2] = red[0];
        out[3] = red[1];
        out[4] = red[2];
        out[5] = red[3];
        out[6] = (double)(*status);
    }
}

// Full FP64 populations of the post-stream state, dense [q][ny][nx].
template <class S, class R, bool FIELD, class P>
__global__ void __launch_bounds__(256) k_read_state(const S* __restrict__ prev, const P* __restrict__ phi,
                                                    Geom gm, Coef<R> c, double* __restrict__ f,
                                                    double* __restrict__ g) {
    const long n = (long)gm.nx * gm.ny;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const int y = (int)(k / gm.nx), x = (int)(k - (long)y * gm.nx);
        R d[9], h[5];
        Drag<R> dr;
        (void)node_state<S, R, FIELD, P>(c, gm, prev, phi, x, y, dr, d, h);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i * n + k] = w9(i) + (double)d[i];
        const double T0 = (double)c.T0;
        g[k] = (double)c.wt0 * T0 + (double)h[0];
#pragma unroll
        for (int j = 1; j < 5; ++j) g[j * n + k] = (double)c.wt1 * T0 + (double)h[j];
    }
}

template <class In, class P>
__global__ void k_convert_phi(const In* __restrict__ in, P* __restrict__ out, Geom gm) {
    const long n = (long)gm.nx * gm.ny;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const int y = (int)(k / gm.nx), x = (int)(k - (long)y * gm.nx);
        if constexpr (sizeof(P) == 2) out[y * gm.pitch + x] = __float2half_rn((float)in[k]);
        else out[y * gm.pitch + x] = (P)in[k];
    }
}

// ---- host launchers ---------------------------------------------------------------

template <class S, class R, class P>
static cudaError_t launch_step_t(const StepLaunch& L, const Coef<R>& c) {
    dim3 blk(L.bx, L.by);
    dim3 grd((L.gm.nx + L.bx - 1) / L.bx, (L.gm.ny + L.by - 1) / L.by);
    if (L.phi)
        k_step<S, R, true, P><<<grd, blk, 0, L.stream>>>((const S*)L.src, (S*)L.dst, (const P*)L.phi,
                                                         L.gm, c, L.status);
    else
        k_step<S, R, false, P><<<grd, blk, 0, L.stream>>>((const S*)L.src, (S*)L.dst, nullptr, L.gm, c,
                                                          L.status);
    return cudaGetLastError();
}

cudaError_t launch_step(const StepLaunch& L, const CoefSet& cs) {
    switch (L.precision) {
        case PREC_F64: return launch_step_t<double, double, double>(L, cs.d);
        case PREC_F32: return launch_step_t<float, float, float>(L, cs.f);
        default: return launch_step_t<__half, float, __half>(L, cs.f);
    }
}

template <class S, class R, class P>
static cudaError_t launch_observe_t(const ObserveLaunch& L, const Coef<R>& c) {
    if (L.phi)
        k_observe<S, R, true, P><<<L.nblocks, 256, 0, L.stream>>>(
            (const S*)L.prev, (const P*)L.phi, L.gm, c, (R*)L.ux, (R*)L.uy, (R*)L.T, (R*)L.p, (R*)L.snap,
            L.snap_valid, L.partials);
    else
        k_observe<S, R, false, P><<<L.nblocks, 256, 0, L.stream>>>(
            (const S*)L.prev, nullptr, L.gm, c, (R*)L.ux, (R*)L.uy, (R*)L.T, (R*)L.p, (R*)L.snap,
            L.snap_valid, L.partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_finish<S, R><<<1, 1024, 0, L.stream>>>((const S*)L.prev, L.gm, c, L.partials, L.nblocks, L.L,
                                             L.dT, L.status, L.out);
    return cudaGetLastError();
}

cudaError_t launch_observe(const ObserveLaunch& L, const CoefSet& cs) {
    switch (L.precision) {
        case PREC_F64: return launch_observe_t<double, double, double>(L, cs.d);
        case PREC_F32: return launch_observe_t<float, float, float>(L, cs.f);
        default: return launch_observe_t<__half, float, __half>(L, cs.f);
    }
}

template <class S, class R>
static cudaError_t launch_nusselt_t(const ObserveLaunch& L, const Coef<R>& c) {
    // npart = 0: only the Nusselt part of the finisher runs
    k_finish<S, R><<<1, 1024, 0, L.stream>>>((const S*)L.prev, L.gm, c, L.partials, 0, L.L, L.dT,
                                             L.status, L.out);
    return cudaGetLastError();
}

cudaError_t launch_nusselt(const ObserveLaunch& L, const CoefSet& cs) {
    switch (L.precision) {
        case PREC_F64: return launch_nusselt_t<double, double>(L, cs.d);
        case PREC_F32: return launch_nusselt_t<float, float>(L, cs.f);
        default: return launch_nusselt_t<__half, float>(L, cs.f);
    }
}

template <class S, class R, class P>
static cudaError_t launch_read_state_t(const ReadStateLaunch& L, const Coef<R>& c) {
    if (L.phi)
        k_read_state<S, R, true, P><<<L.nblocks, 256, 0, L.stream>>>((const S*)L.prev, (const P*)L.phi,
                                                                      L.gm, c, L.f, L.g);
    else
        k_read_state<S, R, false, P><<<L.nblocks, 256, 0, L.stream>>>((const S*)L.prev, nullptr, L.gm, c,
                                                                       L.f, L.g);
    return cudaGetLastError();
}

cudaError_t launch_read_state(const ReadStateLaunch& L, const CoefSet& cs) {
    switch (L.precision) {
        case PREC_F64: return launch_read_state_t<double, double, double>(L, cs.d);
        case PREC_F32: return launch_read_state_t<float, float, float>(L, cs.f);
        default: return launch_read_state_t<__half, float, __half>(L, cs.f);
    }
}

cudaError_t launch_convert_phi(const void* in, int in_is_double, void* out, int precision, const Geom& gm,
                               int nblocks, cudaStream_t s) {
    if (in_is_double) {
        switch (precision) {
            case PREC_F64: k_convert_phi<double, double><<<nblocks, 256, 0, s>>>((const double*)in, (double*)out, gm); break;
            case PREC_F32: k_convert_phi<double, float><<<nblocks, 256, 0, s>>>((const double*)in, (float*)out, gm); break;
            default: k_convert_phi<double, __half><<<nblocks, 256, 0, s>>>((const double*)in, (__half*)out, gm); break;
        }
    } else {
        switch (precision) {
            case PREC_F64: k_convert_phi<float, double><<<nblocks, 256, 0, s>>>((const float*)in, (double*)out, gm); break;
            case PREC_F32: k_convert_phi<float, float><<<nblocks, 256, 0, s>>>((const float*)in, (float*)out, gm); break;
            default: k_convert_phi<float, __half><<<nblocks, 256, 0, s>>>((const float*)in, (__half*)out, gm); break;
        }
    }
    return cudaGetLastError();
}

}  // namespace lbm
