// Run-to-steady-state on the device, and the field extrema used by the
// paper's validation tables (Section 4: Tables 3 and 4 report the maximum
// dimensionless temperature and the maximum stream function).
//
// The steady loop is one CUDA graph: a conditional while-node whose body is
// an even number of step launches followed by a one-block check kernel.  The
// check compares both wall Nusselt numbers (Eq. 38) with the previous check
// and clears the loop condition on convergence, on divergence or at the step
// cap, so the whole run needs a single host synchronisation.
#include <math.h>
#include <string.h>

#include <vector>

#include "lbm_internal.h"

namespace lbm {

// state[0..1]: previous Nu_hot, Nu_cold; [2]: last relative change;
// [3]: checks done; [4]: stop reason (1 converged, 2 diverged, 3 step cap).
template <class T>
__global__ void __launch_bounds__(1024) k_steady_check(Src<T> prev, Geom gm, Coef<typename T::R> c, double L,
                                                       double dT, const int* __restrict__ status, double tol,
                                                       long max_checks, double* __restrict__ state,
                                                       cudaGraphConditionalHandle cond) {
    __shared__ double sh[4 * 32];
    double nh, nc;
    nusselt_block<T>(c, gm, prev, L, dT, sh, &nh, &nc);
    if (threadIdx.x == 0) {
        const long checks = (long)state[3] + 1;
        const double ch = fmax(fabs(nh - state[0]) / fmax(fabs(nh), 1e-300),
                               fabs(nc - state[1]) / fmax(fabs(nc), 1e-300));
        state[0] = nh;
        state[1] = nc;
        state[2] = checks > 1 ? ch : INFINITY;
        state[3] = (double)checks;
        int reason = 0;
        if (*status) reason = 2;
        else if (checks > 1 && ch < tol) reason = 1;
        else if (checks >= max_checks) reason = 3;
        state[4] = (double)reason;
        cudaGraphSetConditional(cond, reason ? 0u : 1u);
    }
}

// One thread per column x: maximum T and the running stream function
// psi(x, y) = sum of trapezoids of u_x along y (psi = 0 on the bottom wall).
template <class T>
__global__ void __launch_bounds__(256) k_extrema(Src<T> prev, const typename T::P* __restrict__ phi, Geom gm,
                                                 Coef<typename T::R> c, double* __restrict__ out) {
    using R = typename T::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= gm.nx) return;
    double tmax = -INFINITY, pmin = 0.0, pmax = 0.0, psi = 0.0, ux_prev = 0.0;
    for (int y = 0; y < gm.ny; ++y) {
        R d[9], h[5];
        Drag<R> dr;
        const Macro<R> mc = phi ? node_state<T, true>(c, gm, prev, phi, x, y, dr, d, h)
                                : node_state<T, false>(c, gm, prev, phi, x, y, dr, d, h);
        const double ux = (double)mc.ux;
        if (y > 0) psi += 0.5 * (ux_prev + ux);
        ux_prev = ux;
        tmax = fmax(tmax, (double)c.T0 + (double)mc.dT);
        pmin = fmin(pmin, psi);
        pmax = fmax(pmax, psi);
    }
    out[3 * x] = tmax;
    out[3 * x + 1] = pmin;
    out[3 * x + 2] = pmax;
}

template <class T> static const Coef<typename T::R>& coef_sel(const CoefSet& cs);
template <> const Coef<double>& coef_sel<PrecF64>(const CoefSet& cs) { return cs.d; }
template <> const Coef<float>& coef_sel<PrecF32Q>(const CoefSet& cs) { return cs.f; }
template <> const Coef<float>& coef_sel<PrecF16>(const CoefSet& cs) { return cs.f; }
template <> const Coef<float>& coef_sel<PrecF32T>(const CoefSet& cs) { return cs.f; }

template <class T>
static cudaError_t launch_check_t(const SteadyCheckLaunch& L, const CoefSet& cs) {
    k_steady_check<T><<<1, 1024, 0, L.stream>>>(src_view<T>(L.prev, L.gm.plane), L.gm, coef_sel<T>(cs), L.L, L.dT,
                                                L.status, L.tol, L.max_checks, L.state, L.cond);
    return cudaGetLastError();
}

cudaError_t launch_steady_check(const SteadyCheckLaunch& L, const CoefSet& cs) {
    switch (L.precision) {
        case PREC_F64: return launch_check_t<PrecF64>(L, cs);
        case PREC_F32: return launch_check_t<PrecF32Q>(L, cs);
        case PREC_F32T: return launch_check_t<PrecF32T>(L, cs);
        default: return launch_check_t<PrecF16>(L, cs);
    }
}

template <class T>
static cudaError_t launch_extrema_t(const void* prev, const void* phi, const Geom& gm, const CoefSet& cs,
                                    double* out, cudaStream_t s) {
    k_extrema<T><<<(gm.nx + 255) / 256, 256, 0, s>>>(src_view<T>(prev, gm.plane), (const typename T::P*)phi, gm,
                                                     coef_sel<T>(cs), out);
    return cudaGetLastError();
}

cudaError_t launch_extrema(int precision, const void* prev, const void* phi, const Geom& gm, const CoefSet& cs,
                           double* out, cudaStream_t s) {
    switch (precision) {
        case PREC_F64: return launch_extrema_t<PrecF64>(prev, phi, gm, cs, out, s);
        case PREC_F32: return launch_extrema_t<PrecF32Q>(prev, phi, gm, cs, out, s);
        case PREC_F32T: return launch_extrema_t<PrecF32T>(prev, phi, gm, cs, out, s);
        default: return launch_extrema_t<PrecF16>(prev, phi, gm, cs, out, s);
    }
}

}  // namespace lbm
