// Batched sweep: many cavities of different size and parameters advanced by
// one persistent kernel launch that runs every requested step, captured once
// into a CUDA graph and replayed.  Each block walks a flat list of tiles
// covering every cavity; a grid-wide barrier separates the steps (each step
// reads the whole previous lattice of its cavity).  The per-node work is the
// same device code as the single-cavity step kernel, so a cavity advanced
// here matches the same cavity advanced alone bit for bit.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "lbm_internal.h"
#include "lbm_sync.cuh"

using namespace lbm;

namespace lbm {

template <class R> struct CavDesc {
    Geom gm;
    void* buf[2];  // B_n / B_{n+1} ping-pong of this cavity
    int ntiles;    // tiles covering this cavity
    Coef<R> c;
};

struct Tile {
    int cav, x0, y0;
};

// Node j of a tile.  lg_tw >= 0: a 2^lg_tw-wide rectangle at (x0, y0), row
// by row; lg_tw < 0: a run of consecutive nodes in the cavity's row-major
// order starting at (x0, y0), wrapping onto the next rows (so tiles leave no
// idle lanes at a cavity's right edge).  Valid when y < ny and x < nx.
__device__ __forceinline__ void tile_node(const Tile& tl, int lg_tw, int j, int nx, int& x, int& y) {
    if (lg_tw >= 0) {
        x = tl.x0 + (j & ((1 << lg_tw) - 1));
        y = tl.y0 + (j >> lg_tw);
    } else {
        x = tl.x0 + j;
        y = tl.y0;
        if (x >= nx) {
            const int q = x / nx;
            y += q;
            x -= q * nx;
        }
    }
}

// The coefficients that differ between the cavities of a sweep follow from
// Ra, Da, the porosity and the size: the viscous and thermal relaxation
// rates (Eq. 20, 31), g beta and the drag coefficients (Eq. 4-5).  cu with
// those fields taken from v.
template <class R>
__host__ __device__ __forceinline__ Coef<R> with_cavity_rates(const Coef<R>& cu, const Coef<R>& v) {
    Coef<R> c = cu;
    c.s[7] = v.s[7];
    c.s[8] = v.s[8];
    c.hs[7] = v.hs[7];
    c.hs[8] = v.hs[8];
    c.z[1] = v.z[1];
    c.z[2] = v.z[2];
    c.hz[1] = v.hz[1];
    c.hz[2] = v.hz[2];
    c.gbeta = v.gbeta;
    c.phi = v.phi;
    c.c_lin = v.c_lin;
    c.c_quad = v.c_quad;
    c.a_lin = v.a_lin;
    c.a_quad = v.a_quad;
    return c;
}

// Split tiles (NPT = 4): a cavity's interior node pairs, (x0, x0 + 1) with
// x0 = 2, 4, ..., 2 npi (npi = floor((nx - 3) / 2): the pairs clear of the
// walls) and 1 <= y <= ny - 2, and its border, every other node: rows 0 and
// ny - 1, then the columns 0, 1 and 2 npi + 2 .. nx - 1 of each inner row
// (the nodes of the pairs that touch a wall).  Border node b of a cavity, by
// that order.
__device__ __forceinline__ void border_node(int b, int nx, int ny, int& x, int& y) {
    if (b < 2 * nx) {
        y = b < nx ? 0 : ny - 1;
        x = b < nx ? b : b - nx;
        return;
    }
    const int npi = (nx - 3) >> 1;
    const int nbc = nx - 2 * npi;  // border columns per inner row: 0, 1 and the right edge
    const int k = b - 2 * nx;
    y = 1 + k / nbc;
    const int col = k - (y - 1) * nbc;
    x = col < 2 ? col : 2 * npi + col;
}
__host__ __device__ constexpr int border_count(int nx, int ny) { return 2 * nx + (ny - 2) * (nx - 2 * ((nx - 3) >> 1)); }

// One tile of one step: tiles hold blockDim.x * NPT nodes (NPT = 3: two
// nodes side by side along x per thread, a run of blockDim.x node pairs in
// the row-major order of the cavity's pairs (x0 even), wrapping onto the next
// rows; a row of odd width ends in a single node.  NPT = 4: split tiles, a
// run of blockDim.x interior pairs (y0 >= 1) or, y0 = -1, of blockDim.x
// border nodes from index x0: the warps of interior tiles never branch into
// the wall rule, which in a small cavity's pair runs would touch every warp).
template <class T, int NPT>
__device__ __forceinline__ void tile_update(const Coef<typename T::R>& c, const Geom& gm, const Src<T>& src,
                                            const Dst<T>& dst, const Tile& tl, int lg_tw, int* status) {
    if constexpr (NPT == 4) {
        if (tl.y0 < 0) {
            const int b = tl.x0 + (int)threadIdx.x;
            if (b < border_count(gm.nx, gm.ny)) {
                int x, y;
                border_node(b, gm.nx, gm.ny, x, y);
                update_node<T, false>(c, gm, src, dst, nullptr, x, y, status);
            }
        } else {
            // the pairs of the inner rows in row-major order, as in pair runs (so a
            // warp's accesses start on the rows' 128-byte boundaries); the lanes
            // whose pair touches a wall idle, the border tiles take those nodes
            const int npx = (gm.nx + 1) >> 1;
            int xp = (tl.x0 >> 1) + (int)threadIdx.x, y = tl.y0;
            if (xp >= npx) {
                const int q = xp / npx;
                y += q;
                xp -= q * npx;
            }
            const int x0 = 2 * xp;
            if (y < gm.ny - 1 && x0 > 0 && x0 + 1 < gm.nx - 1)
                update_xpair<T, false>(c, gm, src, dst, nullptr, x0, y, status);
        }
    } else if constexpr (NPT == 3) {
        const int npx = (gm.nx + 1) >> 1;
        int xp = (tl.x0 >> 1) + (int)threadIdx.x, y = tl.y0;
        if (xp >= npx) {
            const int q = xp / npx;
            y += q;
            xp -= q * npx;
        }
        if (y < gm.ny) update_xpair<T, false>(c, gm, src, dst, nullptr, 2 * xp, y, status);
    } else if constexpr (NPT == 2) {
        int x0, y0, x1, y1;
        tile_node(tl, lg_tw, threadIdx.x, gm.nx, x0, y0);
        tile_node(tl, lg_tw, threadIdx.x + blockDim.x, gm.nx, x1, y1);
        update_pair<T, false>(c, gm, src, dst, nullptr, x0, y0, x0 < gm.nx && y0 < gm.ny, x1, y1,
                              x1 < gm.nx && y1 < gm.ny, status);
    } else {
        int x, y;
        tile_node(tl, lg_tw, threadIdx.x, gm.nx, x, y);
        if (x < gm.nx && y < gm.ny) update_node<T, false>(c, gm, src, dst, nullptr, x, y, status);
    }
}

// One launch runs `nsteps` steps of every cavity.  Buffer parity `par` of
// every cavity holds B_n on entry.  SPLIT (FP32 arithmetic, every cavity's
// other coefficients equal to cu's): the per-cavity rates come from the
// descriptor in shared memory and every other coefficient from the kernel
// parameter cu, which instructions read from the constant bank; without
// SPLIT all come from the descriptor (about 45 values per tile in registers).
// FP32 arithmetic: at most 80 registers (3 blocks of 256 threads, 6 of 128
// per SM); the increment-form collision keeps the pulled values live and its
// node-pair bodies spilled 250-290 bytes under 64.
template <class T, int NPT, bool SPLIT>
__global__ void __launch_bounds__(256, sizeof(typename T::R) == 4 ? 3 : 2)
    k_batch(const CavDesc<typename T::R>* __restrict__ cavs, const Tile* __restrict__ tiles, int ntiles, int lg_tw,
            int dyn, int* __restrict__ tile_ctr, long nsteps, int par, unsigned* bar_count, unsigned* bar_gen,
            long long wait_limit, int* __restrict__ status, int* __restrict__ timeout_flag,
            const Coef<typename T::R> cu) {
    using R = typename T::R;
    __shared__ CavDesc<R> cd;
    __shared__ int chunk_sh;
    constexpr int kChunk = 4;
    // static mode: each block owns a contiguous run of tiles (row-major within a
    // cavity); dynamic mode: blocks take chunks of kChunk tiles from a per-step
    // counter.  Either way the block restages the descriptor only when the
    // cavity changes.
    if (dyn == 2) {
        // dataflow: work items (step, tile) in step-major order from one
        // counter; an item of step s > 0 waits until its cavity has finished
        // step s - 1 (every tile of it was taken earlier by a resident block).
        __shared__ unsigned long long base_sh;
        __shared__ int ok_sh;
        const unsigned long long total = (unsigned long long)nsteps * (unsigned long long)ntiles;
        int cur_cav = -1;
        int ok_cav = -1;        // (cavity, step) whose dependency this block last verified
        long ok_step = -1;
        int pend_cav = -1;      // finished tiles not yet published (thread 0's view)
        int pend_n = 0;
        for (;;) {
            __syncthreads();
            if (threadIdx.x == 0) base_sh = atomicAdd((unsigned long long*)tile_ctr, (unsigned long long)kChunk);
            __syncthreads();
            const unsigned long long base = base_sh;
            if (base >= total) break;
            const unsigned long long end = base + kChunk < total ? base + kChunk : total;
            for (unsigned long long it = base; it < end; ++it) {
                const long sstep = (long)(it / (unsigned long long)ntiles);
                const int t = (int)(it - (unsigned long long)sstep * (unsigned long long)ntiles);
                const Tile tl = tiles[t];
                if (threadIdx.x == 0 && pend_n > 0 && pend_cav != tl.cav) {
                    // publish before waiting on anything else (keeps the progress argument)
                    __threadfence();
                    atomicAdd((int*)&bar_count[2 + pend_cav], pend_n);
                    pend_n = 0;
                }
                if (sstep > 0 && !(tl.cav == ok_cav && sstep == ok_step)) {
                    if (threadIdx.x == 0) {
                        if (pend_n > 0) {
                            __threadfence();
                            atomicAdd((int*)&bar_count[2 + pend_cav], pend_n);
                            pend_n = 0;
                        }
                        const int need = (int)sstep * cavs[tl.cav].ntiles;
                        volatile int* dn = (volatile int*)&bar_count[2 + tl.cav];
                        long long polls = 0;
                        unsigned ns = 32;
                        int ok = 1;
                        while (*dn < need) {
                            if (++polls > wait_limit) {
                                ok = 0;
                                atomicOr(timeout_flag, 1);
                                break;
                            }
                            __nanosleep(ns);
                            ns = ns < 1024 ? 2 * ns : 1024;
                        }
                        __threadfence();
                        ok_sh = ok;
                    }
                    __syncthreads();
                    if (!ok_sh) return;
                    ok_cav = tl.cav;
                    ok_step = sstep;
                }
                if (tl.cav != cur_cav) {
                    __syncthreads();
                    const int* srcw = (const int*)&cavs[tl.cav];
                    int* dstw = (int*)&cd;
                    for (int k = threadIdx.x; k < (int)(sizeof(CavDesc<R>) / sizeof(int)); k += blockDim.x)
                        dstw[k] = srcw[k];
                    __syncthreads();
                    cur_cav = tl.cav;
                }
                const int ps = (par + (int)(sstep & 1)) & 1;
                const Geom gm = cd.gm;
                const Src<T> src = src_view<T>(cd.buf[ps], gm.plane);
                const Dst<T> dst = dst_view<T>(cd.buf[ps ^ 1], gm.plane);
                if constexpr (SPLIT)
                    tile_update<T, NPT>(with_cavity_rates(cu, cd.c), gm, src, dst, tl, lg_tw, &status[tl.cav]);
                else
                    tile_update<T, NPT>(cd.c, gm, src, dst, tl, lg_tw, &status[tl.cav]);
                // the block's stores happen before this barrier; thread 0's GPU-scope
                // fence (cumulative) orders them before the count is published
                __syncthreads();
                if (threadIdx.x == 0) {
                    if (pend_cav != tl.cav) pend_n = 0;
                    pend_cav = tl.cav;
                    ++pend_n;
                }
            }
            if (threadIdx.x == 0 && pend_n > 0) {  // publish at the end of every chunk
                __threadfence();
                atomicAdd((int*)&bar_count[2 + pend_cav], pend_n);
                pend_n = 0;
            }
        }
        return;
    }
    const int per = (ntiles + (int)gridDim.x - 1) / (int)gridDim.x;
    for (long s = 0; s < nsteps; ++s) {
        int cur_cav = -1;
        int t0 = blockIdx.x * per, t1 = min(ntiles, t0 + per);
        for (;;) {
            if (dyn) {
                __syncthreads();
                if (threadIdx.x == 0) chunk_sh = atomicAdd(&tile_ctr[s & 1], kChunk);
                __syncthreads();
                t0 = chunk_sh;
                t1 = min(ntiles, t0 + kChunk);
            }
            if (t0 >= t1) break;
            for (int t = t0; t < t1; ++t) {
                const Tile tl = tiles[t];
                if (tl.cav != cur_cav) {  // block-uniform branch
                    __syncthreads();
                    const int* srcw = (const int*)&cavs[tl.cav];
                    int* dstw = (int*)&cd;
                    for (int k = threadIdx.x; k < (int)(sizeof(CavDesc<R>) / sizeof(int)); k += blockDim.x)
                        dstw[k] = srcw[k];
                    __syncthreads();
                    cur_cav = tl.cav;
                }
                const Geom gm = cd.gm;
                const Src<T> src = src_view<T>(cd.buf[par], gm.plane);
                const Dst<T> dst = dst_view<T>(cd.buf[par ^ 1], gm.plane);
                if constexpr (SPLIT)
                    tile_update<T, NPT>(with_cavity_rates(cu, cd.c), gm, src, dst, tl, lg_tw, &status[tl.cav]);
                else
                    tile_update<T, NPT>(cd.c, gm, src, dst, tl, lg_tw, &status[tl.cav]);
            }
            if (!dyn) break;
        }
        par ^= 1;
        if (s + 1 < nsteps) {
            __threadfence();
            // the releasing block clears the counter of step s + 1 (used two steps ago)
            if (!grid_barrier(bar_count, bar_gen, gridDim.x, wait_limit, timeout_flag, &tile_ctr[(s + 1) & 1])) return;
        }
    }
}

// Mean Nusselt numbers (Eq. 38) of every cavity, one block per cavity, FP64.
template <class T>
__global__ void __launch_bounds__(256) k_batch_nusselt(const CavDesc<typename T::R>* __restrict__ cavs,
                                                       int prev_par, const double* __restrict__ Ls,
                                                       double* __restrict__ out) {
    using R = typename T::R;
    __shared__ double sh[2][32];
    const CavDesc<R>& cd = cavs[blockIdx.x];
    const Geom gm = cd.gm;
    const Src<T> prev = src_view<T>(cd.buf[prev_par], gm.plane);
    const double L = Ls[2 * blockIdx.x], dT = Ls[2 * blockIdx.x + 1];
    double wl = 0.0, wr = 0.0;
    for (int y = threadIdx.x; y < gm.ny; y += blockDim.x) {
        double tl[5], tr[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            tl[k] = (double)node_dT<T>(cd.c, gm, prev, k, y);
            tr[k] = (double)node_dT<T>(cd.c, gm, prev, gm.nx - 1 - k, y);
        }
        const double dl = (-25.0 * tl[0] + 48.0 * tl[1] - 36.0 * tl[2] + 16.0 * tl[3] - 3.0 * tl[4]) / 12.0;
        const double dr = (25.0 * tr[0] - 48.0 * tr[1] + 36.0 * tr[2] - 16.0 * tr[3] + 3.0 * tr[4]) / 12.0;
        const double wt = (y == 0 || y == gm.ny - 1) ? 0.5 : 1.0;
        wl += wt * (-L * dl / dT);
        wr += wt * (-L * dr / dT);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        wl += __shfl_xor_sync(0xffffffffu, wl, o);
        wr += __shfl_xor_sync(0xffffffffu, wr, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][warp] = wl;
        sh[1][warp] = wr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += sh[0][w];
            b += sh[1][w];
        }
        out[2 * blockIdx.x] = a / (double)(gm.ny - 1);
        out[2 * blockIdx.x + 1] = b / (double)(gm.ny - 1);
    }
}

}  // namespace lbm

// ---------------------------------------------------------------------------------

namespace {

constexpr long long kDefaultWaitPolls = 20000000;  // ~2-20 s of 100 ns polls

// th = 0: linear tiles, runs of tw consecutive nodes in row-major order
struct TuneChoice {
    int tw = 128, th = 2, blocks_per_sm = 0, dyn = 0;
};

// th = -1: runs of tw node pairs (two nodes side by side along x per thread);
// th = -2: split tiles, runs of tw interior pairs or tw border nodes
int tile_nodes(const TuneChoice& t) { return t.th < 0 ? 2 * t.tw : (t.th == 0 ? t.tw : t.tw * t.th); }

// Tiles of 256 or 512 nodes run with 256-thread blocks; tiles of 32 or 64
// nodes with one-warp blocks, whose block synchronisation is a warp's.
int block_of(const TuneChoice& t) { return t.th < 0 ? t.tw : (tile_nodes(t) >= 256 ? 256 : 32); }

}  // namespace

struct lbm_batch_s {
    int ncav = 0;
    int precision = LBM_F32;
    std::vector<lbm_params> params;
    std::vector<Derived> dv;
    std::vector<Geom> gm;
    std::vector<CoefSet> coef;
    std::vector<size_t> off[2];
    std::vector<int> cav_tiles;
    size_t pool_bytes = 0;
    void* pool = nullptr;
    void* descs = nullptr;  // CavDesc<R>[ncav]
    Tile* tiles = nullptr;
    int ntiles = 0;
    double* Ls = nullptr;   // (L, dT) per cavity
    double* nu_dev = nullptr;
    int* status = nullptr;  // per cavity
    int* timeout_flag = nullptr;
    unsigned* bar = nullptr;  // count, gen, then one finished-tile counter per cavity
    int* tile_ctr = nullptr;  // dynamic: one counter per step parity; dataflow: one 64-bit item counter
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int par = 0;  // parity holding B_n
    long t = 0;
    TuneChoice tune;
    bool split = false;  // k_batch<T, NPT, true>: batch-wide coefficients from the constant bank
    int nblocks = 0;
    long long wait_limit = kDefaultWaitPolls;
    cudaGraphExec_t gexec = nullptr;
    long gexec_steps = 0;
    int gexec_par = -1;
    long long gexec_limit = -1;
    std::string err;
    std::string signature;
};

namespace {

int bfail(lbm_batch b, int code, const std::string& m) {
    if (b) b->err = m;
    else set_global_error(m);
    return code;
}

#define BCK(b, expr)                                                                     \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T, bool SPLIT> const void* kernel_ptr(int npt) {
    switch (npt) {
        case 4: return (const void*)&k_batch<T, 4, SPLIT>;
        case 3: return (const void*)&k_batch<T, 3, SPLIT>;
        case 2: return (const void*)&k_batch<T, 2, SPLIT>;
        default: return (const void*)&k_batch<T, 1, SPLIT>;
    }
}

// FP64 keeps every coefficient in the descriptor: with the split its
// two-node body spills.
const void* batch_kernel(int precision, int npt, bool split) {
    if (precision == LBM_F64) return kernel_ptr<PrecF64P, false>(npt);
    if (precision == LBM_F32_FRAMED)
        return split ? kernel_ptr<PrecF32TP, true>(npt) : kernel_ptr<PrecF32TP, false>(npt);
    return split ? kernel_ptr<PrecF32QP, true>(npt) : kernel_ptr<PrecF32QP, false>(npt);
}

int npt_of(const TuneChoice& t) { return t.th == -2 ? 4 : t.th == -1 ? 3 : (tile_nodes(t) == 2 * block_of(t) ? 2 : 1); }

int log2i(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

template <class R> int upload_descs(lbm_batch b);

int build_tiles(lbm_batch b) {
    if (b->stream) BCK(b, cudaStreamSynchronize(b->stream));  // queued launches may still read the old list
    std::vector<Tile> tl;
    b->cav_tiles.assign(b->ncav, 0);
    for (int c = 0; c < b->ncav; ++c) {
        const int nx = b->gm[c].nx, ny = b->gm[c].ny;
        if (b->tune.th == -2) {
            // the pairs of the inner rows (those clear of the walls run there), then the border nodes
            const long npx = (nx + 1) / 2;
            for (long p0 = 0; p0 < npx * (ny - 2); p0 += b->tune.tw) {
                tl.push_back(Tile{c, (int)(2 * (p0 % npx)), (int)(1 + p0 / npx)});
                ++b->cav_tiles[c];
            }
            for (long b0 = 0; b0 < border_count(nx, ny); b0 += b->tune.tw) {
                tl.push_back(Tile{c, (int)b0, -1});
                ++b->cav_tiles[c];
            }
        } else if (b->tune.th == -1) {
            const long npx = (nx + 1) / 2;
            for (long p0 = 0; p0 < npx * ny; p0 += b->tune.tw) {
                tl.push_back(Tile{c, (int)(2 * (p0 % npx)), (int)(p0 / npx)});
                ++b->cav_tiles[c];
            }
        } else if (b->tune.th == 0) {
            for (long k0 = 0; k0 < (long)nx * ny; k0 += b->tune.tw) {
                tl.push_back(Tile{c, (int)(k0 % nx), (int)(k0 / nx)});
                ++b->cav_tiles[c];
            }
        } else {
            for (int y0 = 0; y0 < ny; y0 += b->tune.th)
                for (int x0 = 0; x0 < nx; x0 += b->tune.tw) {
                    tl.push_back(Tile{c, x0, y0});
                    ++b->cav_tiles[c];
                }
        }
    }
    if (b->tiles) cudaFree(b->tiles);
    b->tiles = nullptr;
    b->ntiles = (int)tl.size();
    BCK(b, cudaMalloc(&b->tiles, sizeof(Tile) * tl.size()));
    BCK(b, cudaMemcpy(b->tiles, tl.data(), sizeof(Tile) * tl.size(), cudaMemcpyHostToDevice));
    if (b->descs) return b->precision == LBM_F64 ? upload_descs<double>(b) : upload_descs<float>(b);
    return LBM_OK;
}

int grid_size(lbm_batch b, int* nblocks) {
    int dev = 0, nsm = 0, per_sm = 0;
    BCK(b, cudaGetDevice(&dev));
    BCK(b, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const void* k = batch_kernel(b->precision, npt_of(b->tune), b->split);
    BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block_of(b->tune), 0));
    if (per_sm < 1) return bfail(b, LBM_ERR_CUDA, "batched kernel cannot be resident");
    int want = b->tune.blocks_per_sm > 0 ? std::min(b->tune.blocks_per_sm, per_sm) : per_sm;
    *nblocks = std::max(1, std::min(nsm * want, b->ntiles));
    return LBM_OK;
}

int launch(lbm_batch b, long nsteps, int par, cudaStream_t s) {
    void* args[14];
    long ns = nsteps;
    int pr = par;
    unsigned* cnt = b->bar;
    unsigned* gen = b->bar + 1;
    long long lim = b->wait_limit;
    int lg = b->tune.th <= 0 ? -1 : log2i(b->tune.tw), nt = b->ntiles;
    const void* descs = b->descs;
    const Tile* tiles = b->tiles;
    int dyn = b->tune.dyn;
    args[0] = &descs;
    args[1] = &tiles;
    args[2] = &nt;
    args[3] = &lg;
    args[4] = &dyn;
    args[5] = &b->tile_ctr;
    args[6] = &ns;
    args[7] = &pr;
    args[8] = &cnt;
    args[9] = &gen;
    args[10] = &lim;
    args[11] = &b->status;
    args[12] = &b->timeout_flag;
    Coef<float> cuf = b->coef[0].f;  // the batch-wide coefficients (SPLIT kernels read them)
    Coef<double> cud = b->coef[0].d;
    args[13] = b->precision == LBM_F64 ? (void*)&cud : (void*)&cuf;
    cudaError_t ez = cudaMemsetAsync(b->tile_ctr, 0, 2 * sizeof(int), s);
    if (ez == cudaSuccess && b->tune.dyn == 2)  // finished-tile counters of the dataflow mode
        ez = cudaMemsetAsync(b->bar + 2, 0, sizeof(unsigned) * (size_t)b->ncav, s);
    if (ez != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("counter reset: ") + cudaGetErrorString(ez));
    const int npt = npt_of(b->tune);
    const void* k = batch_kernel(b->precision, npt, b->split);
    cudaError_t e = cudaLaunchCooperativeKernel(k, dim3(b->nblocks), dim3(block_of(b->tune)), args, 0, s);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("cooperative launch: ") + cudaGetErrorString(e));
    return LBM_OK;
}

template <class R> int upload_descs(lbm_batch b) {
    std::vector<CavDesc<R>> h(b->ncav);
    for (int c = 0; c < b->ncav; ++c) {
        h[c].gm = b->gm[c];
        h[c].buf[0] = (char*)b->pool + b->off[0][c];
        h[c].buf[1] = (char*)b->pool + b->off[1][c];
        h[c].ntiles = c < (int)b->cav_tiles.size() ? b->cav_tiles[c] : 0;
        if constexpr (sizeof(R) == 8) h[c].c = b->coef[c].d;
        else h[c].c = b->coef[c].f;
    }
    // the split kernels need every coefficient but the per-cavity rates equal
    // across the batch, bit for bit
    bool split = sizeof(R) == 4;
    for (int c = 1; c < b->ncav && split; ++c) {
        const Coef<R> x = with_cavity_rates(h[0].c, h[c].c);
        split = memcmp(&x, &h[c].c, sizeof(Coef<R>)) == 0;
    }
    b->split = split;
    if (!b->descs) BCK(b, cudaMalloc(&b->descs, sizeof(CavDesc<R>) * b->ncav));
    BCK(b, cudaMemcpy(b->descs, h.data(), sizeof(CavDesc<R>) * b->ncav, cudaMemcpyHostToDevice));
    return LBM_OK;
}

// Rest state in both buffers of every cavity, then one step (S_0 -> B_0).
int reset(lbm_batch b) {
    BCK(b, cudaMemsetAsync(b->pool, 0, b->pool_bytes, b->stream));
    BCK(b, cudaMemsetAsync(b->status, 0, sizeof(int) * b->ncav, b->stream));
    BCK(b, cudaMemsetAsync(b->timeout_flag, 0, sizeof(int), b->stream));
    BCK(b, cudaMemsetAsync(b->bar, 0, 2 * sizeof(unsigned), b->stream));
    int rc = launch(b, 1, 0, b->stream);
    if (rc != LBM_OK) return rc;
    b->par = 1;
    b->t = 0;
    return LBM_OK;
}

void drop_graph(lbm_batch b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->gexec_steps = 0;
    b->gexec_par = -1;
}

int run_steps(lbm_batch b, long nsteps, cudaStream_t s) {
    if (nsteps <= 0) return LBM_OK;
    const int par = b->par;
    if (!(b->gexec && b->gexec_steps == nsteps && b->gexec_par == par && b->gexec_limit == b->wait_limit)) {
        drop_graph(b);
        cudaGraph_t g = nullptr;
        BCK(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = launch(b, nsteps, par, b->cap_stream);
        cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
        if (rc != LBM_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e2 != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e2));
        cudaError_t e = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        b->gexec_steps = nsteps;
        b->gexec_par = par;
        b->gexec_limit = b->wait_limit;
    }
    BCK(b, cudaGraphLaunch(b->gexec, s));
    if (nsteps & 1) b->par ^= 1;
    return LBM_OK;
}

std::string device_name() {
    int dev = 0;
    cudaDeviceProp pr;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return "unknown";
    std::string n = pr.name;
    std::replace(n.begin(), n.end(), ' ', '_');
    return n;
}

// Autotuner cache: one line per (signature) -> "tw th blocks_per_sm".
bool cache_lookup(const std::string& path, const std::string& sig, TuneChoice* tc) {
    std::ifstream in(path);
    std::string line;
    while (std::getline(in, line)) {
        std::istringstream ss(line);
        std::string key;
        TuneChoice t;
        if (ss >> key >> t.tw >> t.th >> t.blocks_per_sm >> t.dyn && key == sig) {
            *tc = t;
            return true;
        }
    }
    return false;
}

void cache_store(const std::string& path, const std::string& sig, const TuneChoice& tc) {
    std::ofstream out(path, std::ios::app);
    if (out) out << sig << " " << tc.tw << " " << tc.th << " " << tc.blocks_per_sm << " " << tc.dyn << "\n";
}

}  // namespace

extern "C" {

int lbm_batch_init(const lbm_params* p, int ncav, void* stream, lbm_batch* out) {
    if (!out) return bfail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!p || ncav <= 0) return bfail(nullptr, LBM_ERR_ARG, "need at least one cavity");
    const int prec = p[0].precision;
    if (prec != LBM_F32 && prec != LBM_F64 && prec != LBM_F32_FRAMED)
        return bfail(nullptr, LBM_ERR_ARG, "batched cavities run in LBM_F32, LBM_F32_FRAMED or LBM_F64");
    lbm_batch b = new lbm_batch_s();
    b->ncav = ncav;
    b->precision = prec;
    b->params.assign(p, p + ncav);
    b->dv.resize(ncav);
    b->gm.resize(ncav);
    b->coef.resize(ncav);
    b->off[0].resize(ncav);
    b->off[1].resize(ncav);
    b->stream = (cudaStream_t)stream;
    std::ostringstream sig;
    sig << device_name() << ":p" << prec << ":n" << ncav;
    unsigned long long hsh = 1469598103934665603ull;
    size_t at = 0;
    for (int c = 0; c < ncav; ++c) {
        std::string why;
        if (p[c].precision != prec) {
            delete b;
            return bfail(nullptr, LBM_ERR_ARG, "every cavity of a batch needs the same precision");
        }
        if (p[c].use_phi_field) {
            delete b;
            return bfail(nullptr, LBM_ERR_ARG, "batched cavities use uniform porosity");
        }
        int rc = setup_lattice(&p[c], &b->dv[c], &b->coef[c], &b->gm[c], &why);
        if (rc != LBM_OK) {
            delete b;
            return bfail(nullptr, rc, "cavity " + std::to_string(c) + ": " + why);
        }
        const size_t bb = (state_buffer_bytes(prec, b->gm[c].plane) + 255) / 256 * 256;
        b->off[0][c] = at;
        b->off[1][c] = at + bb;
        at += 2 * bb;
        hsh = (hsh ^ (unsigned long long)(p[c].nx * 65537 + p[c].ny)) * 1099511628211ull;
    }
    sig << ":h" << std::hex << hsh;
    b->signature = sig.str();
    b->pool_bytes = at;
    cudaError_t e = cudaSuccess;
#define BI(expr)                                                    \
    do {                                                            \
        e = (expr);                                                 \
        if (e != cudaSuccess) {                                     \
            std::string m_ = std::string(#expr) + ": " + cudaGetErrorString(e); \
            lbm_batch_destroy(b);                                   \
            return bfail(nullptr, LBM_ERR_CUDA, m_);                \
        }                                                           \
    } while (0)
    BI(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    BI(cudaMalloc(&b->pool, b->pool_bytes));
    BI(cudaMalloc(&b->status, sizeof(int) * ncav));
    BI(cudaMalloc(&b->timeout_flag, sizeof(int)));
    BI(cudaMalloc(&b->bar, (2 + (size_t)ncav) * sizeof(unsigned)));
    BI(cudaMalloc(&b->tile_ctr, 2 * sizeof(int)));
    BI(cudaMalloc(&b->Ls, sizeof(double) * 2 * ncav));
    BI(cudaMalloc(&b->nu_dev, sizeof(double) * 2 * ncav));
#undef BI
    std::vector<double> Ls(2 * ncav);
    for (int c = 0; c < ncav; ++c) {
        Ls[2 * c] = b->dv[c].L;
        Ls[2 * c + 1] = b->dv[c].dT;
    }
    int rc = LBM_OK;
    if (cudaMemcpy(b->Ls, Ls.data(), sizeof(double) * 2 * ncav, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = bfail(b, LBM_ERR_CUDA, "parameter upload");
    if (rc == LBM_OK) rc = prec == LBM_F64 ? upload_descs<double>(b) : upload_descs<float>(b);
    if (rc == LBM_OK) rc = build_tiles(b);
    if (rc == LBM_OK) rc = grid_size(b, &b->nblocks);
    if (rc == LBM_OK) rc = reset(b);
    if (rc != LBM_OK) {
        std::string m = b->err;
        lbm_batch_destroy(b);
        return bfail(nullptr, rc, m);
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch b, long nsteps) {
    TraceRange trace_("lbm_batch_step");
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    if (nsteps < 0) return bfail(b, LBM_ERR_ARG, "nsteps < 0");
    // one launch runs at most 2^16 steps: the dataflow mode's per-cavity
    // finished-tile counters (steps x tiles of a cavity) stay within 32 bits
    constexpr long kMaxStepsPerLaunch = 1L << 16;
    for (long left = nsteps; left > 0;) {
        const long k = left < kMaxStepsPerLaunch ? left : kMaxStepsPerLaunch;
        int rc = run_steps(b, k, b->stream);
        if (rc != LBM_OK) return rc;
        b->t += k;
        left -= k;
    }
    return LBM_OK;
}

int lbm_batch_nusselt(lbm_batch b, double* nu_hot, double* nu_cold) {
    TraceRange trace_("lbm_batch_nusselt");
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    const int prev = b->par ^ 1;
    if (b->precision == LBM_F64)
        k_batch_nusselt<PrecF64P><<<b->ncav, 256, 0, b->stream>>>((const CavDesc<double>*)b->descs, prev, b->Ls,
                                                                 b->nu_dev);
    else if (b->precision == LBM_F32_FRAMED)
        k_batch_nusselt<PrecF32TP><<<b->ncav, 256, 0, b->stream>>>((const CavDesc<float>*)b->descs, prev, b->Ls,
                                                                  b->nu_dev);
    else
        k_batch_nusselt<PrecF32QP><<<b->ncav, 256, 0, b->stream>>>((const CavDesc<float>*)b->descs, prev, b->Ls,
                                                                 b->nu_dev);
    BCK(b, cudaGetLastError());
    std::vector<double> h(2 * b->ncav);
    BCK(b, cudaMemcpyAsync(h.data(), b->nu_dev, sizeof(double) * 2 * b->ncav, cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    for (int c = 0; c < b->ncav; ++c) {
        if (nu_hot) nu_hot[c] = h[2 * c];
        if (nu_cold) nu_cold[c] = h[2 * c + 1];
    }
    return LBM_OK;
}

int lbm_batch_status(lbm_batch b, int* status) {
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    std::vector<int> h(b->ncav);
    int to = 0;
    BCK(b, cudaMemcpyAsync(h.data(), b->status, sizeof(int) * b->ncav, cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaMemcpyAsync(&to, b->timeout_flag, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    int any = 0;
    for (int c = 0; c < b->ncav; ++c) {
        if (status) status[c] = h[c] ? LBM_ERR_DIVERGED : LBM_OK;
        any |= h[c];
    }
    if (to) return bfail(b, LBM_ERR_TIMEOUT, "a grid-barrier wait ran out; the lattice state is incomplete");
    if (any) return bfail(b, LBM_ERR_DIVERGED, "at least one cavity raised its divergence flag");
    return LBM_OK;
}

int lbm_batch_read_state(lbm_batch b, int cav, double* f_dev, double* g_dev) {
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    if (cav < 0 || cav >= b->ncav || !f_dev || !g_dev) return bfail(b, LBM_ERR_ARG, "bad cavity or output");
    ReadStateLaunch L;
    L.precision = b->precision;
    L.prev = (char*)b->pool + b->off[b->par ^ 1][cav];
    L.phi = nullptr;
    L.gm = b->gm[cav];
    L.f = f_dev;
    L.g = g_dev;
    L.nblocks = kReduceBlocks;
    L.stream = b->stream;
    BCK(b, launch_read_state(L, b->coef[cav]));
    return LBM_OK;
}

int lbm_batch_set_wait_limit(lbm_batch b, long long polls) {
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    if (polls < 0) return bfail(b, LBM_ERR_ARG, "polls < 0");
    b->wait_limit = polls;
    BCK(b, cudaMemsetAsync(b->timeout_flag, 0, sizeof(int), b->stream));
    BCK(b, cudaMemsetAsync(b->bar, 0, 2 * sizeof(unsigned), b->stream));
    return LBM_OK;
}

int lbm_batch_tune(lbm_batch b, const char* cache_path, int* tile_w, int* tile_h, int* blocks_per_sm) {
    TraceRange trace_("lbm_batch_tune");
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    TuneChoice best;
    bool cached = cache_path && cache_lookup(cache_path, b->signature, &best);
    if (!cached) {
        const int shapes[][2] = {{32, 8}, {64, 4}, {128, 2}, {256, 1}, {64, 8}, {128, 4}, {256, 2}, {512, 1},
                                 {32, 1}, {32, 2}, {64, 1}, {32, 0}, {64, 0}, {256, 0}, {512, 0},
                                 {32, -1}, {64, -1}, {128, -1}, {256, -1}, {32, -2}, {64, -2}, {128, -2}, {256, -2}};
        const int occ[] = {0, 2};
        float best_ms = 1e30f;
        cudaEvent_t e0, e1;
        BCK(b, cudaEventCreate(&e0));
        BCK(b, cudaEventCreate(&e1));
        const long nsteps = 20;
        for (auto& sh : shapes)
            for (int o : occ)
            for (int dyn = 0; dyn < 3; ++dyn) {
                b->tune.tw = sh[0];
                b->tune.th = sh[1];
                b->tune.blocks_per_sm = o;
                b->tune.dyn = dyn;
                int rc = build_tiles(b);
                if (rc == LBM_OK) rc = grid_size(b, &b->nblocks);
                drop_graph(b);
                if (rc == LBM_OK) rc = run_steps(b, 2, b->stream);  // warm
                if (rc != LBM_OK) return rc;
                BCK(b, cudaEventRecord(e0, b->stream));
                rc = run_steps(b, nsteps, b->stream);
                if (rc != LBM_OK) return rc;
                BCK(b, cudaEventRecord(e1, b->stream));
                BCK(b, cudaEventSynchronize(e1));
                float ms = 0.f;
                BCK(b, cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best_ms) {
                    best_ms = ms;
                    best = b->tune;
                }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (cache_path) cache_store(cache_path, b->signature, best);
    }
    b->tune = best;
    int rc = build_tiles(b);
    if (rc == LBM_OK) rc = grid_size(b, &b->nblocks);
    drop_graph(b);
    if (rc == LBM_OK) rc = reset(b);  // tuning advanced the lattices: start again from t = 0
    if (rc != LBM_OK) return rc;
    if (tile_w) *tile_w = best.tw;
    if (tile_h) *tile_h = best.th;
    if (blocks_per_sm) *blocks_per_sm = best.blocks_per_sm;
    return LBM_OK;
}

int lbm_batch_set_tiles(lbm_batch b, int tile_w, int tile_h, int blocks_per_sm, int dynamic) {
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    const int tn = tile_h == 0 ? tile_w : tile_w * tile_h;
    const bool pairs = (tile_h == -1 || tile_h == -2) && (tile_w == 32 || tile_w == 64 || tile_w == 128 || tile_w == 256);
    if (!pairs && (tile_w <= 0 || tile_h < 0 || (tn != 32 && tn != 64 && tn != 256 && tn != 512) ||
                   (tile_h > 0 && ((tile_w & (tile_w - 1)) != 0 || tile_w < 32)) || blocks_per_sm < 0))
        return bfail(b, LBM_ERR_ARG, "tiles hold 32, 64, 256 or 512 nodes: a power-of-two width >= 32 times "
                                     "tile_h rows, tile_h = 0 for runs of tile_w consecutive nodes, or "
                                     "tile_h = -1 for runs of tile_w (32 to 256) node pairs, -2 for the same "
                                     "over each cavity's interior with its border in runs of its own");
    if (blocks_per_sm < 0) return bfail(b, LBM_ERR_ARG, "blocks_per_sm < 0");
    b->tune.tw = tile_w;
    b->tune.th = tile_h;
    b->tune.blocks_per_sm = blocks_per_sm;
    b->tune.dyn = dynamic < 0 || dynamic > 2 ? 0 : dynamic;
    int rc = build_tiles(b);
    if (rc == LBM_OK) rc = grid_size(b, &b->nblocks);
    drop_graph(b);
    if (rc == LBM_OK) rc = reset(b);
    return rc;
}

int lbm_batch_query(lbm_batch b, long* t, int* ntiles, int* nblocks) {
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    if (t) *t = b->t;
    if (ntiles) *ntiles = b->ntiles;
    if (nblocks) *nblocks = b->nblocks;
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch b) {
    if (!b) return LBM_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    if (b->pool) cudaFree(b->pool);
    if (b->descs) cudaFree(b->descs);
    if (b->tiles) cudaFree(b->tiles);
    if (b->Ls) cudaFree(b->Ls);
    if (b->nu_dev) cudaFree(b->nu_dev);
    if (b->status) cudaFree(b->status);
    if (b->timeout_flag) cudaFree(b->timeout_flag);
    if (b->bar) cudaFree(b->bar);
    if (b->tile_ctr) cudaFree(b->tile_ctr);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
    return LBM_OK;
}

const char* lbm_batch_last_error(lbm_batch b) { return b ? b->err.c_str() : lbm_last_error(nullptr); }

}  // extern "C"
