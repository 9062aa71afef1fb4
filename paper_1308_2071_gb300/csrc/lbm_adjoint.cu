// Discrete adjoint of the time stepping: gradient of the mean Nusselt number
// of the hot wall (Eq. 38) after N steps with respect to a per-cell porosity
// field, by reverse sweeps with checkpoint-and-recompute.
//
// Notation: B_k is the post-collision lattice after step k (B_{-1} = rest),
// S_N = pull(B_{N-1}) + wall rule, J = Nu_hot(S_N).  The adjoint state
// M^(k)(x) = dJ / d(populations pulled into node x at step k) lives on nodes;
// dJ/dB_k(y)_i = M^(k)_i(y + e_i) is gathered (the reverse of the pull, read
// over reversed directions, so no atomics).  A wall node uses the pulled
// populations of its inner neighbour, so a fluid node also folds in the
// reverse of the wall nodes that extrapolate from it.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "lbm_adjoint.cuh"
#include "lbm_internal.h"

using namespace lbm;

namespace lbm {

// dJ/dS_N as the initial adjoint state: J depends on T at the columns 1..4
// next to the hot wall (the wall column is the imposed T_h); on first-order
// adiabatic walls T(x, 0) = T(x, 1) and T(x, ny-1) = T(x, ny-2).
template <class R>
__global__ void k_adj_seed(R* __restrict__ M, Geom gm, double L, double dT) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y < 1 || y > gm.ny - 2) return;
    const double cx[5] = {-25.0, 48.0, -36.0, 16.0, -3.0};
    double wy = 1.0;
    if (gm.thermal_bc == 0) {
        if (y == 1) wy += 0.5;
        if (y == gm.ny - 2) wy += 0.5;
    }
    for (int x = 1; x <= 4 && x <= gm.nx - 2; ++x) {
        const double a = -L * cx[x] / (12.0 * dT * (double)(gm.ny - 1)) * wy;
        for (int j = 0; j < 5; ++j) M[(9 + j) * gm.plane + y * gm.pitch + x] = (R)a;
    }
}

template <class R>
__device__ __forceinline__ void gather_adjoint(const R* __restrict__ M, const Geom& gm, int x, int y, R (&lf)[9],
                                               R (&lh)[5]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int xs = x + ex9(i), ys = y + ey9(i);
        const bool in = xs >= 0 && xs < gm.nx && ys >= 0 && ys < gm.ny;
        lf[i] = in ? M[i * gm.plane + ys * gm.pitch + xs] : R(0);
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int xs = x + ex9(j), ys = y + ey9(j);
        const bool in = xs >= 0 && xs < gm.nx && ys >= 0 && ys < gm.ny;
        lh[j] = in ? M[(9 + j) * gm.plane + ys * gm.pitch + xs] : R(0);
    }
}

// The populations pulled into node off, as deviations from the rest state:
// with framed storage the thermal values are re-expressed relative to T0
// (the frame is an exact change of variables of the stored values, so the
// adjoint of the step is the one of the plain deviations).
template <class T>
__device__ __forceinline__ void pull_rest(const Coef<typename T::R>& c, const Src<T>& src, const Geom& gm, int off,
                                          typename T::R (&d)[9], typename T::R (&h)[5]) {
    pull<T>(src, gm, off, d, h);
    if constexpr (Framed<T>::value) {
        const typename T::R F = frame_in<T>(c, src, gm, off, h);
        h[0] += c.wt0 * F;
#pragma unroll
        for (int j = 1; j < 5; ++j) h[j] += c.wt1 * F;
    }
}

__device__ __forceinline__ bool wall_is_dirichlet(const Geom& gm, Normal nr) {
    return gm.thermal_bc == 1 || nr.dx != 0;
}

template <class R>
__device__ __forceinline__ R wall_dT(const Coef<R>& c, const Geom& gm, int x) {
    return gm.thermal_bc == 1 ? c.dTc : (x == 0 ? c.dTh : c.dTc);
}

// Reverse of one node for one step: from M^(k+1) and the forward input B_k
// to M^(k) at (x, y), adding this step's porosity sensitivity to gphi.
// RING = false: (x, y) is at least two nodes from every wall, so it is a
// fluid node and no wall node extrapolates from it.
template <class T, bool RING>
__device__ __forceinline__ void adjoint_node(const Src<T>& state, const typename T::R* __restrict__ Mnext,
                                             typename T::R* __restrict__ Mcur, const typename T::P* __restrict__ phi,
                                             double* __restrict__ gphi, const Geom& gm, const Coef<typename T::R>& c,
                                             int x, int y) {
    using R = typename T::R;
    const int off = y * gm.pitch + x;
    const long k = (long)y * gm.nx + x;
    const Normal nr = normal_of(gm, x, y);
    R lf[9], lh[5];
    if (RING && (nr.dx != 0 || nr.dy != 0)) {
        // wall node: it reads no pulled populations of its own; its porosity
        // sensitivity is computed here, its inner neighbour's by that node
#pragma unroll
        for (int q = 0; q < NPOP; ++q) Mcur[q * gm.plane + off] = R(0);
        gather_adjoint<R>(Mnext, gm, x, y, lf, lh);
        const int xf = x + nr.dx, yf = y + nr.dy, offf = yf * gm.pitch + xf;
        R df[9], hf[5];
        pull_rest<T>(c, state, gm, offf, df, hf);
        Tape<R> tf;
        tape_node<R>(c, (R)phi[offf], df, hf, tf);
        R dfb[9] = {R(0)}, hfb[5] = {R(0)}, pfb = R(0);
        const R pb = wall_node_adjoint<R>(c, tf, (R)phi[off], wall_is_dirichlet(gm, nr), wall_dT<R>(c, gm, x), lf, lh,
                                          dfb, hfb, pfb);
        gphi[k] += (double)pb;
        return;
    }
    gather_adjoint<R>(Mnext, gm, x, y, lf, lh);
    R d[9], h[5];
    pull_rest<T>(c, state, gm, off, d, h);
    Tape<R> t;
    tape_node<R>(c, (R)phi[off], d, h, t);
    R db[9] = {R(0)}, hb[5] = {R(0)}, pb = R(0);
    fluid_node_adjoint<R>(c, t, lf, lh, db, hb, pb);
    // wall nodes b = x - n whose inward normal n points at this node
    if (RING)
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            if (dx == 0 && dy == 0) continue;
            const int xb = x - dx, yb = y - dy;
            const Normal nb = normal_of(gm, xb, yb);
            if (nb.dx != dx || nb.dy != dy) continue;
            R lfb[9], lhb[5];
            gather_adjoint<R>(Mnext, gm, xb, yb, lfb, lhb);
            (void)wall_node_adjoint<R>(c, t, (R)phi[yb * gm.pitch + xb], wall_is_dirichlet(gm, nb),
                                       wall_dT<R>(c, gm, xb), lfb, lhb, db, hb, pb);
        }
#pragma unroll
    for (int i = 0; i < 9; ++i) Mcur[i * gm.plane + off] = db[i];
#pragma unroll
    for (int j = 0; j < 5; ++j) Mcur[(9 + j) * gm.plane + off] = hb[j];
    gphi[k] += (double)pb;
}

// One reverse step over the interior nodes (two or more nodes from every
// wall), grid-stride over a grid sized to the resident capacity.
template <class T>
__global__ void __launch_bounds__(256, sizeof(typename T::R) == 4 ? 4 : 1)
    k_adjoint(Src<T> state, const typename T::R* __restrict__ Mnext, typename T::R* __restrict__ Mcur,
              const typename T::P* __restrict__ phi, double* __restrict__ gphi, Geom gm, Coef<typename T::R> c) {
    const int w = gm.nx - 4;
    const long n = (long)w * (gm.ny - 4);
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const int yi = (int)(k / w);
        adjoint_node<T, false>(state, Mnext, Mcur, phi, gphi, gm, c, 2 + (int)(k - (long)yi * w), 2 + yi);
    }
}

// The same over the ring of nodes within two of a wall (nx, ny >= 5): rows
// 0, 1, ny-2, ny-1 in full, then columns 0, 1, nx-2, nx-1 of rows 2..ny-3.
template <class T>
__global__ void __launch_bounds__(64)
    k_adjoint_ring(Src<T> state, const typename T::R* __restrict__ Mnext, typename T::R* __restrict__ Mcur,
                   const typename T::P* __restrict__ phi, double* __restrict__ gphi, Geom gm,
                   Coef<typename T::R> c) {
    const long rows = 4L * gm.nx, n = rows + 4L * (gm.ny - 4);
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        int x, y;
        if (k < rows) {
            const int r = (int)(k / gm.nx);
            x = (int)(k - (long)r * gm.nx);
            y = r < 2 ? r : gm.ny - 4 + r;
        } else {
            const int j = (int)(k - rows), r = j >> 2, q = j & 3;
            y = 2 + r;
            x = q < 2 ? q : gm.nx - 4 + q;
        }
        adjoint_node<T, true>(state, Mnext, Mcur, phi, gphi, gm, c, x, y);
    }
}

template <class Out>
__global__ void k_adj_out(const double* __restrict__ g, Out* __restrict__ out, long n) {
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
        out[k] = (Out)g[k];
}

}  // namespace lbm

namespace {

// Second stream for the ring kernel, and the two events that join it with
// the main stream around every reverse step.
struct RingStream {
    cudaStream_t s2 = nullptr;
    cudaEvent_t main_done = nullptr, ring_done = nullptr;
    cudaError_t init() {
        cudaError_t e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&main_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ring_done, cudaEventDisableTiming);
        return e;
    }
    ~RingStream() {
        if (ring_done) cudaEventDestroy(ring_done);
        if (main_done) cudaEventDestroy(main_done);
        if (s2) cudaStreamDestroy(s2);  // resources go once its work is done
    }
};

// Third stream for the recomputation of the next segment, with an event per
// half of the segment storage for "recomputed" and for "read by the reverse
// sweep" (both recorded once at the start, so the first waits pass).
struct RecomputeStream {
    cudaStream_t s3 = nullptr;
    cudaEvent_t ready[2] = {nullptr, nullptr}, free[2] = {nullptr, nullptr}, end = nullptr;
    cudaError_t init(cudaStream_t main) {
        cudaError_t e = cudaStreamCreateWithFlags(&s3, cudaStreamNonBlocking);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            e = cudaEventCreateWithFlags(&ready[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&free[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventRecord(free[k], main);  // after the set-up on the main stream
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&end, cudaEventDisableTiming);
        return e;
    }
    // an event behind all recompute work (the main stream waits for it before it returns)
    cudaEvent_t done() {
        return cudaEventRecord(end, s3) == cudaSuccess ? end : ready[0];
    }
    ~RecomputeStream() {
        if (end) cudaEventDestroy(end);
        for (int k = 0; k < 2; ++k) {
            if (ready[k]) cudaEventDestroy(ready[k]);
            if (free[k]) cudaEventDestroy(free[k]);
        }
        if (s3) cudaStreamDestroy(s3);
    }
};

template <class T>
cudaError_t adjoint_sweep(const AdjointJob& J) {
    using R = typename T::R;
    const Geom& gm = J.gm;
    const Coef<R>& c = *(const Coef<R>*)J.coef;
    const int N = (int)J.nsteps, K = (int)J.ckpt_every;
    const size_t buf = J.buf_bytes;
    const size_t mbytes = (size_t)gm.plane * NPOP * sizeof(R);
    cudaStream_t s = J.stream;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e0 == cudaSuccess) e0 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adjoint<T>, 256, 0);
    if (e0 != cudaSuccess) return e0;
    const long inner = (long)(gm.nx - 4) * (gm.ny - 4), ring = 4L * gm.nx + 4L * (gm.ny - 4);
    // one interior node per thread: the hardware starts the blocks of the
    // next wave as blocks finish (a grid-stride loop over fewer resident
    // blocks ran its last pass with a fifth of the threads busy)
    (void)per_sm;
    const int nblk = (int)std::max(1L, (inner + 255) / 256);
    const int nring = (int)std::max(1L, std::min((long)nsm, (ring + 63) / 64));
    const int nseg = (N + K - 1) / K;
    R* M[2] = {(R*)J.madj, (R*)J.madj + (size_t)gm.plane * NPOP};
    cudaError_t e = cudaMemsetAsync(M[0], 0, mbytes, s);
    if (e != cudaSuccess) return e;
    k_adj_seed<R><<<(gm.ny + 255) / 256, 256, 0, s>>>(M[0], gm, J.L, J.dT);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(J.gphi, 0, sizeof(double) * (size_t)gm.nx * gm.ny, s)) != cudaSuccess) return e;
    // Within a reverse step the ring and interior nodes are independent (each
    // writes its own nodes of M^(k) and gphi), so the ring kernel runs on a
    // second stream beside the interior kernel; the main stream waits for it
    // before the next step.  The recomputation of a segment needs only its
    // checkpoint, so it runs on a third stream into the other half of the
    // segment storage while the main stream reverses the segment after it:
    // the latency-bound forward steps and reverse steps overlap.
    RingStream rs;
    if ((e = rs.init()) != cudaSuccess) return e;
    auto join = [&]() { return cudaStreamWaitEvent(s, rs.ring_done, 0); };
    if ((e = cudaEventRecord(rs.ring_done, rs.s2)) != cudaSuccess) return e;  // nothing pending on s2 yet
    RecomputeStream rc;
    if ((e = rc.init(s)) != cudaSuccess) return e;
    CoefSet cs;
    if (sizeof(R) == 8) cs.d = *(const Coef<double>*)J.coef;
    else cs.f = *(const Coef<float>*)J.coef;
    const size_t half = (size_t)(K > 1 ? K - 1 : 0) * buf;  // bytes of one half of the segment storage
    auto seg_len = [&](int sg) { return (N - sg * K) < K ? (N - sg * K) : K; };
    auto slot_of = [&](int sg, int hf, int m) -> const void* {
        return m == 0 ? (const char*)J.ckpt + (size_t)sg * buf : (const char*)J.seg + hf * half + (size_t)(m - 1) * buf;
    };
    // recompute segment sg into half hf on the third stream, once the reverse
    // sweep that last read that half is done
    auto recompute = [&](int sg, int hf) -> cudaError_t {
        cudaError_t er = cudaStreamWaitEvent(rc.s3, rc.free[hf], 0);
        for (int m = 1; m < seg_len(sg) && er == cudaSuccess; ++m) {
            StepLaunch L;
            L.precision = J.precision;
            L.src = slot_of(sg, hf, m - 1);
            L.dst = (void*)slot_of(sg, hf, m);
            L.phi = J.phi;
            L.gm = gm;
            L.bx = J.bx;
            L.by = J.by;
            L.npt = J.npt;
            L.status = J.status;
            L.stream = rc.s3;
            L.pdl = m > 1;  // directly behind the previous recomputing step
            er = launch_step(L, cs);
        }
        if (er == cudaSuccess) er = cudaEventRecord(rc.ready[hf], rc.s3);
        return er;
    };
    int a = 0, hf = 0;
    e = recompute(nseg - 1, 0);
    for (int sg = nseg - 1; sg >= 0 && e == cudaSuccess; --sg, hf ^= 1) {
        const int j0 = sg * K, len = seg_len(sg);
        if (sg > 0 && (e = recompute(sg - 1, hf ^ 1)) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(s, rc.ready[hf], 0)) != cudaSuccess) break;
        for (int j = j0 + len - 1; j >= j0; --j) {
            const Src<T> st = src_view<T>(slot_of(sg, hf, j - j0), gm.plane);
            // main_done: everything before this step (previous step, recompute) has finished on s
            if ((e = cudaEventRecord(rs.main_done, s)) != cudaSuccess) break;
            if ((e = cudaStreamWaitEvent(rs.s2, rs.main_done, 0)) != cudaSuccess) break;
            k_adjoint_ring<T><<<nring, 64, 0, rs.s2>>>(st, M[a], M[a ^ 1], (const typename T::P*)J.phi, J.gphi,
                                                        gm, c);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            if ((e = cudaEventRecord(rs.ring_done, rs.s2)) != cudaSuccess) break;
            k_adjoint<T><<<nblk, 256, 0, s>>>(st, M[a], M[a ^ 1], (const typename T::P*)J.phi, J.gphi, gm, c);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            if ((e = join()) != cudaSuccess) break;
            a ^= 1;
        }
        // the half is free again once this segment's reverse sweep is done
        if (e == cudaSuccess) e = cudaEventRecord(rc.free[hf], s);
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, rc.done(), 0);
    if (e != cudaSuccess) {
        (void)join();  // leave no ring work behind the main stream's back
        return e;
    }
    const long n = (long)gm.nx * gm.ny;
    if (sizeof(R) == 8) k_adj_out<double><<<kReduceBlocks, 256, 0, s>>>(J.gphi, (double*)J.out, n);
    else k_adj_out<float><<<kReduceBlocks, 256, 0, s>>>(J.gphi, (float*)J.out, n);
    return cudaGetLastError();
}

}  // namespace

namespace lbm {
cudaError_t launch_adjoint_sweep(const AdjointJob& J) {
    if (J.precision == PREC_F64) return adjoint_sweep<PrecF64>(J);
    if (J.precision == PREC_F32T) return adjoint_sweep<PrecF32T>(J);
    return adjoint_sweep<PrecF32Q>(J);
}
}  // namespace lbm
