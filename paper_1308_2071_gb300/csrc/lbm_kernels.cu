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
//
// Launched as a programmatic dependent of the previous step (back-to-back
// steps of small lattices), a block starts while that step drains and waits
// here until it has completed and its writes are visible: the step reads the
// whole previous lattice and rewrites the buffer the previous step read.
// Without that launch attribute the wait returns at once.
__device__ __forceinline__ void wait_for_previous_step() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// OBS: an observing step, which also stores the temperatures of the node
// columns next to the vertical walls into obs (obs_put) for the Nusselt
// number of the new state; otherwise obs is unused.
template <class T, bool FIELD, bool OBS>
__global__ void __launch_bounds__(256) k_step(Src<T> src, Dst<T> dst, const typename T::P* __restrict__ phi,
                                              Geom gm, Coef<typename T::R> c, int* __restrict__ status,
                                              double* __restrict__ obs) {
    wait_for_previous_step();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= gm.nx || y >= gm.ny) return;
    update_node<T, FIELD, OBS>(c, gm, src, dst, phi, x, y, status, obs);
}

// Two nodes per thread, (x, y) and (x, y + blockDim.y): when both are fluid
// nodes all 28 loads are issued before any arithmetic, doubling the bytes in
// flight per thread (the FP16-flow variant moves 38 B per node, too few to
// cover HBM latency with one node per thread).  Wall nodes take the general
// path one at a time.
// FP32 arithmetic: at most 64 registers (4 blocks of 256 threads, 8 of 128
// per SM), which measured faster than the unconstrained 68-80 registers at
// every size and storage type: more warps keep more loads in flight.  FP64
// would spill under that limit.
template <class T, bool FIELD, bool OBS>
__global__ void __launch_bounds__(256, sizeof(typename T::R) == 4 ? 4 : 1)
    k_step2(Src<T> src, Dst<T> dst, const typename T::P* __restrict__ phi, Geom gm, Coef<typename T::R> c,
            int* __restrict__ status, double* __restrict__ obs) {
    wait_for_previous_step();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y0 = blockIdx.y * (2 * blockDim.y) + threadIdx.y;
    const int y1 = y0 + blockDim.y;
    if (x >= gm.nx || y0 >= gm.ny) return;
    update_pair<T, FIELD, OBS>(c, gm, src, dst, phi, x, y0, true, x, y1, y1 < gm.ny, status, obs);
}

// Two nodes per thread side by side, (x0, y) and (x0 + 1, y) with x0 even:
// the populations with e_x = 0 are loaded, and every population stored, as
// aligned pairs (8-byte FP32, 4-byte FP16 accesses), a third fewer memory
// instructions than two nodes apart along y.  Same register cap.
template <class T, bool FIELD, bool OBS>
__global__ void __launch_bounds__(256, sizeof(typename T::R) == 4 ? 4 : 1)
    k_step2x(Src<T> src, Dst<T> dst, const typename T::P* __restrict__ phi, Geom gm, Coef<typename T::R> c,
             int* __restrict__ status, double* __restrict__ obs) {
    wait_for_previous_step();
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x0 >= gm.nx || y >= gm.ny) return;
    update_xpair<T, FIELD, OBS>(c, gm, src, dst, phi, x0, y, status, obs);
}

// ---- observables ------------------------------------------------------------------

// Macroscopic fields of the post-stream state S_n, rebuilt by pulling from
// B_{n-1} and applying the wall rule, plus per-block partials (FP64) of
// max|u|, max|u - u_prev|, sum of population deviations, sum of T - T0.
template <class T, bool FIELD>
__global__ void __launch_bounds__(256) k_observe(Src<T> prev, const typename T::P* __restrict__ phi, Geom gm,
                                                 Coef<typename T::R> c, typename T::R* ux_out,
                                                 typename T::R* uy_out, typename T::R* T_out,
                                                 typename T::R* p_out, typename T::R* snap, int snap_valid,
                                                 double* __restrict__ partials) {
    using R = typename T::R;
    __shared__ double sh[4 * 32];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const long n = (long)gm.nx * gm.ny;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const int y = (int)(k / gm.nx), x = (int)(k - (long)y * gm.nx);
        R d[9], h[5];
        Drag<R> dr;
        const Macro<R> mc = node_state<T, FIELD>(c, gm, prev, phi, x, y, dr, d, h);
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
        v[0] = fmax_nan(v[0], (double)mc.umag);
        v[1] = fmax_nan(v[1], du);
        v[2] += (double)sd;
        v[3] += (double)mc.dT;
    }
    block_reduce4(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) partials[blockIdx.x * 4 + k] = v[k];
    }
}

// One block: folds the per-block partials in a fixed order and evaluates the
// mean Nusselt numbers (Eq. 38) of both vertical walls, FP64 throughout:
// Nu(y) = -L dT/dx / dT with the one-sided five-point derivative
// (-25 T0 + 48 T1 - 36 T2 + 16 T3 - 3 T4) / 12, trapezoidal mean over y.
// out[0..6] = nu_hot, nu_cold, max|u|, max|du|, sum d, sum (T - T0), status.
template <class T>
__global__ void __launch_bounds__(1024) k_finish(Src<T> prev, Geom gm, Coef<typename T::R> c,
                                                 const double* __restrict__ partials, int npart, double L,
                                                 double dT, const int* __restrict__ status,
                                                 double* __restrict__ out) {
    __shared__ double sh[4 * 32];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < npart; b += blockDim.x) {
        v[0] = fmax_nan(v[0], partials[4 * b]);
        v[1] = fmax_nan(v[1], partials[4 * b + 1]);
        v[2] += partials[4 * b + 2];
        v[3] += partials[4 * b + 3];
    }
    block_reduce4(v, sh);
    __syncthreads();
    const double red[4] = {v[0], v[1], v[2], v[3]};
    double nh, nc;
    nusselt_block<T>(c, gm, prev, L, dT, sh, &nh, &nc);
    if (threadIdx.x == 0) {
        out[0] = nh;
        out[1] = nc;
        out[2] = red[0];
        out[3] = red[1];
        out[4] = red[2];
        out[5] = red[3];
        out[6] = (double)(*status);
    }
}

// Row-parallel mean Nusselt numbers (Eq. 38): one thread per wall row in
// one-warp blocks (so the rows' scattered loads spread over many SMs), warp
// sums into partials; the last block to finish folds the partials in a fixed
// order (deterministic), writes out[0..1] and re-arms the counter.  OBS: the
// temperatures come from the wall columns the step before stored (obs_dT),
// else they are pulled from B_{n-1} (node_dT); both give the same values.
template <class T, bool OBS>
__global__ void __launch_bounds__(32) k_nusselt_rows(Src<T> prev, const double* __restrict__ obs, Geom gm,
                                                     Coef<typename T::R> c, double L, double dT,
                                                     double* __restrict__ partials, unsigned* __restrict__ counter,
                                                     double* __restrict__ out) {
    __shared__ bool last;
    double a = 0.0, b = 0.0;
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y < gm.ny) {
        double tl[5], tr[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            if constexpr (OBS) {
                tl[k] = obs_dT<T>(c, gm, obs, k, y);
                tr[k] = obs_dT<T>(c, gm, obs, 5 + k, y);
            } else {
                tl[k] = (double)node_dT<T>(c, gm, prev, k, y);
                tr[k] = (double)node_dT<T>(c, gm, prev, gm.nx - 1 - k, y);
            }
        }
        const double dl = (-25.0 * tl[0] + 48.0 * tl[1] - 36.0 * tl[2] + 16.0 * tl[3] - 3.0 * tl[4]) / 12.0;
        const double dr = (25.0 * tr[0] - 48.0 * tr[1] + 36.0 * tr[2] - 16.0 * tr[3] + 3.0 * tr[4]) / 12.0;
        const double wt = (y == 0 || y == gm.ny - 1) ? 0.5 : 1.0;
        a = wt * (-L * dl / dT);
        b = wt * (-L * dr / dT);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    a = 0.0;
    b = 0.0;
    for (unsigned k = threadIdx.x; k < gridDim.x; k += 32) {
        a += __ldcg(partials + 2 * k);
        b += __ldcg(partials + 2 * k + 1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (threadIdx.x == 0) {
        out[0] = a / (double)(gm.ny - 1);
        out[1] = b / (double)(gm.ny - 1);
        *counter = 0u;
    }
}

// Full FP64 populations of the post-stream state, dense [q][ny][nx].
template <class T, bool FIELD>
__global__ void __launch_bounds__(256) k_read_state(Src<T> prev, const typename T::P* __restrict__ phi, Geom gm,
                                                    Coef<typename T::R> c, double* __restrict__ f,
                                                    double* __restrict__ g) {
    using R = typename T::R;
    const long n = (long)gm.nx * gm.ny;
    // rest weights in FP64 (Eq. 37 first occurrence), independent of the arithmetic type
    const double varpi = (double)c.varpi, T0 = (double)c.T0;
    const double wt0 = (1.0 - varpi) / 5.0, wt1 = (4.0 + varpi) / 20.0;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const int y = (int)(k / gm.nx), x = (int)(k - (long)y * gm.nx);
        R d[9], h[5];
        Drag<R> dr;
        const Macro<R> mc = node_state<T, FIELD>(c, gm, prev, phi, x, y, dr, d, h);
        // framed storage: h is relative to T0 + F (F = 0 otherwise)
        const double Tr = Framed<T>::value ? T0 + (double)mc.F : T0;
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i * n + k] = w9(i) + (double)d[i];
        g[k] = wt0 * Tr + (double)h[0];
#pragma unroll
        for (int j = 1; j < 5; ++j) g[j * n + k] = wt1 * Tr + (double)h[j];
    }
}

// Counts the cells of a porosity field outside the open interval (0, 1)
// (NaN included) into *bad.
template <class In>
__global__ void k_count_bad_phi(const In* __restrict__ in, long n, unsigned long long* __restrict__ bad) {
    unsigned long long c = 0;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const In v = in[k];
        c += (v > In(0) && v < In(1)) ? 0ull : 1ull;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(bad, c);
}

template <class In, class P>
__global__ void k_convert_phi(const In* __restrict__ in, P* __restrict__ out, Geom gm) {
    const long n = (long)gm.nx * gm.ny;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const int y = (int)(k / gm.nx), x = (int)(k - (long)y * gm.nx);
        out[y * gm.pitch + x] = (P)in[k];
    }
}

// ---- host launchers ---------------------------------------------------------------

template <class T> static const Coef<typename T::R>& coef_of(const CoefSet& cs);
template <> const Coef<double>& coef_of<PrecF64>(const CoefSet& cs) { return cs.d; }
template <> const Coef<float>& coef_of<PrecF32Q>(const CoefSet& cs) { return cs.f; }
template <> const Coef<float>& coef_of<PrecF16>(const CoefSet& cs) { return cs.f; }
template <> const Coef<float>& coef_of<PrecF32T>(const CoefSet& cs) { return cs.f; }

// Launches kernel k with the step's arguments, as a programmatic dependent of
// the previous work on the stream when L.pdl is set.
template <class T, class K>
static cudaError_t launch_one_step(K k, dim3 grd, dim3 blk, const StepLaunch& L, const Src<T>& s, const Dst<T>& d,
                                   const typename T::P* phi, const Coef<typename T::R>& c) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grd;
    cfg.blockDim = blk;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = L.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = L.pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, s, d, phi, L.gm, c, L.status, L.obs);
}

template <class T, bool FIELD, bool OBS>
static cudaError_t launch_step_k(const StepLaunch& L, const CoefSet& cs) {
    dim3 blk(L.bx, L.by);
    const Src<T> s = src_view<T>(L.src, L.gm.plane);
    const Dst<T> d = dst_view<T>(L.dst, L.gm.plane);
    const typename T::P* phi = FIELD ? (const typename T::P*)L.phi : nullptr;
    if (L.npt == 2) {
        dim3 grd2((L.gm.nx + L.bx - 1) / L.bx, (L.gm.ny + 2 * L.by - 1) / (2 * L.by));
        return launch_one_step<T>(k_step2<T, FIELD, OBS>, grd2, blk, L, s, d, phi, coef_of<T>(cs));
    }
    if (L.npt == 3) {
        dim3 grdx((L.gm.nx + 2 * L.bx - 1) / (2 * L.bx), (L.gm.ny + L.by - 1) / L.by);
        return launch_one_step<T>(k_step2x<T, FIELD, OBS>, grdx, blk, L, s, d, phi, coef_of<T>(cs));
    }
    dim3 grd((L.gm.nx + L.bx - 1) / L.bx, (L.gm.ny + L.by - 1) / L.by);
    return launch_one_step<T>(k_step<T, FIELD, OBS>, grd, blk, L, s, d, phi, coef_of<T>(cs));
}

template <class T>
static cudaError_t launch_step_t(const StepLaunch& L, const CoefSet& cs) {
    if (L.obs) return L.phi ? launch_step_k<T, true, true>(L, cs) : launch_step_k<T, false, true>(L, cs);
    return L.phi ? launch_step_k<T, true, false>(L, cs) : launch_step_k<T, false, false>(L, cs);
}

template <class T>
static cudaError_t launch_observe_t(const ObserveLaunch& L, const CoefSet& cs) {
    using R = typename T::R;
    const Src<T> s = src_view<T>(L.prev, L.gm.plane);
    if (L.phi)
        k_observe<T, true><<<L.nblocks, 256, 0, L.stream>>>(s, (const typename T::P*)L.phi, L.gm, coef_of<T>(cs),
                                                            (R*)L.ux, (R*)L.uy, (R*)L.T, (R*)L.p, (R*)L.snap,
                                                            L.snap_valid, L.partials);
    else
        k_observe<T, false><<<L.nblocks, 256, 0, L.stream>>>(s, nullptr, L.gm, coef_of<T>(cs), (R*)L.ux,
                                                             (R*)L.uy, (R*)L.T, (R*)L.p, (R*)L.snap,
                                                             L.snap_valid, L.partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_finish<T><<<1, 1024, 0, L.stream>>>(s, L.gm, coef_of<T>(cs), L.partials, L.nblocks, L.L, L.dT, L.status,
                                          L.out);
    return cudaGetLastError();
}

template <class T>
static cudaError_t launch_nusselt_t(const ObserveLaunch& L, const CoefSet& cs) {
    // partials holds 2 doubles per block; counter is zero between launches
    const int nb = (L.gm.ny + 31) / 32;
    const Src<T> s = src_view<T>(L.prev, L.gm.plane);
    if (L.obs)
        k_nusselt_rows<T, true><<<nb, 32, 0, L.stream>>>(s, L.obs, L.gm, coef_of<T>(cs), L.L, L.dT, L.partials,
                                                         L.counter, L.out);
    else
        k_nusselt_rows<T, false><<<nb, 32, 0, L.stream>>>(s, nullptr, L.gm, coef_of<T>(cs), L.L, L.dT, L.partials,
                                                          L.counter, L.out);
    return cudaGetLastError();
}

template <class T>
static cudaError_t launch_read_state_t(const ReadStateLaunch& L, const CoefSet& cs) {
    const Src<T> s = src_view<T>(L.prev, L.gm.plane);
    if (L.phi)
        k_read_state<T, true><<<L.nblocks, 256, 0, L.stream>>>(s, (const typename T::P*)L.phi, L.gm,
                                                               coef_of<T>(cs), L.f, L.g);
    else
        k_read_state<T, false><<<L.nblocks, 256, 0, L.stream>>>(s, nullptr, L.gm, coef_of<T>(cs), L.f, L.g);
    return cudaGetLastError();
}

#define LBM_DISPATCH(prec, fn, ...)                     \
    switch (prec) {                                     \
        case PREC_F64: return fn<PrecF64>(__VA_ARGS__); \
        case PREC_F32: return fn<PrecF32Q>(__VA_ARGS__); \
        case PREC_F32T: return fn<PrecF32T>(__VA_ARGS__); \
        default: return fn<PrecF16>(__VA_ARGS__);       \
    }

cudaError_t launch_step(const StepLaunch& L, const CoefSet& cs) { LBM_DISPATCH(L.precision, launch_step_t, L, cs) }
cudaError_t launch_observe(const ObserveLaunch& L, const CoefSet& cs) {
    LBM_DISPATCH(L.precision, launch_observe_t, L, cs)
}
cudaError_t launch_nusselt(const ObserveLaunch& L, const CoefSet& cs) {
    LBM_DISPATCH(L.precision, launch_nusselt_t, L, cs)
}
cudaError_t launch_read_state(const ReadStateLaunch& L, const CoefSet& cs) {
    LBM_DISPATCH(L.precision, launch_read_state_t, L, cs)
}

size_t state_buffer_bytes(int precision, int plane) {
    switch (precision) {
        case PREC_F64: return buffer_bytes<PrecF64>(plane);
        case PREC_F32: return buffer_bytes<PrecF32Q>(plane);
        case PREC_F32T: return buffer_bytes<PrecF32T>(plane);
        default: return buffer_bytes<PrecF16>(plane);
    }
}

size_t phi_bytes(int precision, int plane) {
    return (size_t)plane * (precision == PREC_F64 ? sizeof(double) : sizeof(float));
}

cudaError_t launch_count_bad_phi(const void* in, int in_is_double, long n, unsigned long long* bad, int nblocks,
                                 cudaStream_t s) {
    if (in_is_double) k_count_bad_phi<double><<<nblocks, 256, 0, s>>>((const double*)in, n, bad);
    else k_count_bad_phi<float><<<nblocks, 256, 0, s>>>((const float*)in, n, bad);
    return cudaGetLastError();
}

cudaError_t launch_convert_phi(const void* in, int in_is_double, void* out, int precision, const Geom& gm,
                               int nblocks, cudaStream_t s) {
    const bool to_double = precision == PREC_F64;
    if (in_is_double) {
        if (to_double) k_convert_phi<double, double><<<nblocks, 256, 0, s>>>((const double*)in, (double*)out, gm);
        else k_convert_phi<double, float><<<nblocks, 256, 0, s>>>((const double*)in, (float*)out, gm);
    } else {
        if (to_double) k_convert_phi<float, double><<<nblocks, 256, 0, s>>>((const float*)in, (double*)out, gm);
        else k_convert_phi<float, float><<<nblocks, 256, 0, s>>>((const float*)in, (float*)out, gm);
    }
    return cudaGetLastError();
}

}  // namespace lbm
