// Device building blocks of the coupled D2Q9 / D2Q5 MRT lattice Boltzmann step
// (Liu, He, Li, Tao, arXiv:1308.2071, Section 3) on the side-heated cavity of
// Section 4.
//
// Populations are held as deviations from the rest state of the initial
// condition: d_i = f_i - w_i rho0 (D2Q9) and h_j = g_j - w~_j T0 (D2Q5).  The
// model is affine in that shift (sum_i e_i w_i = 0, M w rho0 = rho0 (1, -2, 1,
// 0, ...), N w~ T0 = T0 (1, 0, 0, varpi, 0)), so every formula below is the
// paper's formula minus its value at rest, with rho0 = 1 and delta_t = 1
// (Section 4).  Deviations are O(Ma^2) and O(Delta T), which keeps FP32 and
// FP16 storage accurate.
//
// Storage layout (structure of arrays): plane q of a buffer holds population
// q for every node, row-major with x fastest and a row pitch (in elements)
// that makes every row start on a 128-byte boundary; planes 0..8 are f
// (Eq. 8 order: rest, E, N, W, S, NE, NW, SW, SE), planes 9..13 are g (Eq. 26
// order: rest, E, N, W, S).  Flow and thermal planes may use different
// storage types (see PrecF16); both use the same pitch in elements.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lbm {

// ---- lattice -----------------------------------------------------------------

// D2Q9 velocity components of Eq. 8 (c = 1).
__host__ __device__ constexpr int ex9(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}
__host__ __device__ constexpr int ey9(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
}
// D2Q9 weights (stated after Eq. 13).
__host__ __device__ constexpr double w9(int i) {
    return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}
// D2Q5 velocities of Eq. 26 are the first five D2Q9 velocities.

constexpr int NPOP = 14;  // 9 flow + 5 thermal planes per buffer

// ---- storage conversions ------------------------------------------------------

// CG = false: read-only (non-coherent) cached loads, for buffers never
// written during the launch.  CG = true: coherent loads (ld.global.ca), for
// kernels that read data other blocks of the same launch wrote (the
// persistent batched kernel): a weak load observes every write that happens
// before it through the kernel's release/acquire synchronisation (the grid
// barrier, or the dataflow schedule's wait), and may hit L1, which the
// neighbouring nodes' shifted pulls and frames reuse; the non-coherent path
// of __ldg gives no such guarantee within a launch.
template <class S, class R, bool CG = false> struct Conv;
template <bool CG> struct Conv<double, double, CG> {
    static __device__ __forceinline__ double ld(const double* p) { return CG ? __ldca(p) : __ldg(p); }
    static __device__ __forceinline__ void st(double* p, double v) { *p = v; }
};
template <bool CG> struct Conv<float, float, CG> {
    static __device__ __forceinline__ float ld(const float* p) { return CG ? __ldca(p) : __ldg(p); }
    static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
};
template <bool CG> struct Conv<__half, float, CG> {
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(CG ? __ldca(p) : __ldg(p)); }
    static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
};

// Two nodes side by side along x, starting at an even x: every row starts on
// a 128-byte boundary, so the pair is one aligned 2-element access.
template <class S, class R, bool CG = false> struct Conv2;
template <bool CG> struct Conv2<double, double, CG> {
    static __device__ __forceinline__ double2 ld(const double* p) {
        return CG ? __ldca((const double2*)p) : __ldg((const double2*)p);
    }
    static __device__ __forceinline__ void st(double* p, double a, double b) { *(double2*)p = make_double2(a, b); }
};
template <bool CG> struct Conv2<float, float, CG> {
    static __device__ __forceinline__ float2 ld(const float* p) {
        return CG ? __ldca((const float2*)p) : __ldg((const float2*)p);
    }
    static __device__ __forceinline__ void st(float* p, float a, float b) { *(float2*)p = make_float2(a, b); }
};
template <bool CG> struct Conv2<__half, float, CG> {
    static __device__ __forceinline__ float2 ld(const __half* p) {
        return __half22float2(CG ? __ldca((const __half2*)p) : __ldg((const __half2*)p));
    }
    static __device__ __forceinline__ void st(__half* p, float a, float b) { *(__half2*)p = __floats2half2_rn(a, b); }
};

// ---- precision variants -----------------------------------------------------------
// SF: storage of the nine flow planes, SG: storage of the five thermal planes,
// R: arithmetic, P: storage of a per-cell porosity field.
struct PrecF64 {
    using SF = double;
    using SG = double;
    using R = double;
    using P = double;
    static constexpr bool cg = false;
};
struct PrecF32 {
    using SF = float;
    using SG = float;
    using R = float;
    using P = float;
    static constexpr bool cg = false;
};
// Storage with a per-node temperature frame: one more plane holds F(x), the
// node's T - T0 when the node was last written, rounded to the frame's
// storage type ST, and the thermal planes hold g_j - w~_j (T0 + F(x)) instead
// of g_j - w~_j T0.  The stored thermal values are then the small
// non-equilibrium parts, so FP32 resolves the per-step change of T even where
// |T - T0| is near 1/2 (about 1e-8 per step on a 1024^2 lattice, against the
// 3e-8 spacing of FP32 numbers near 0.3, where plain deviations lose it).
//
// PrecF32T: the frame in FP32.  PrecF32Q: the frame as an 8-bit integer k,
// F = k fq with fq a power of two (Coef::fq), so that F(x) - F(x') and the
// frame change of a node are exact in FP32 and the frame costs one byte per
// node each way.  The remainder |T - T0 - F| <= fq / 2 is then small enough
// that FP32 keeps the slow evolution (checked against FP64 over 50,000 steps).
struct PrecF32T : PrecF32 {
    static constexpr bool framed = true;
    using ST = float;
};
struct PrecF32Q : PrecF32 {
    static constexpr bool framed = true;
    using ST = int8_t;
};
// FP16 flow deviations (|d| stays near 1e-2, where half rounds to ~4e-6) with
// FP32 thermal deviations relative to the 8-bit frame of PrecF32Q (thermal
// deviations reach w~_0 (T_h - T0) = 0.3 at the hot wall, where half would
// round to ~1.2e-4 and drift the temperature field).
struct PrecF16 {
    using SF = __half;
    using SG = float;
    using R = float;
    using P = float;
    static constexpr bool cg = false;
    static constexpr bool paired = true;  // update_pair computes both nodes with paired FP32 instructions
    static constexpr bool framed = true;
    using ST = int8_t;
};
// Increment-form collision (see collide) for the FP32 storage variants.
template <class T> struct IncForm {
    static constexpr bool value = std::is_same<typename T::R, float>::value && std::is_same<typename T::SF, float>::value;
};
template <class T, class = void> struct Paired {
    static constexpr bool value = false;
};
template <class T> struct Paired<T, decltype((void)T::paired)> {
    static constexpr bool value = T::paired;
};
template <class T, class = void> struct Framed {
    static constexpr bool value = false;
};
template <class T> struct Framed<T, decltype((void)T::framed)> {
    static constexpr bool value = T::framed;
};
// Storage type of the frame plane (the thermal type when there is none).
template <class T, class = void> struct FrameStore {
    using type = typename T::SG;
};
template <class T> struct FrameStore<T, decltype((void)sizeof(typename T::ST))> {
    using type = typename T::ST;
};

// Same arithmetic, L2-only loads (persistent kernels).
struct PrecF64P : PrecF64 {
    static constexpr bool cg = true;
};
struct PrecF32P : PrecF32 {
    static constexpr bool cg = true;
};
struct PrecF32TP : PrecF32P {
    static constexpr bool framed = true;
    using ST = float;
};
struct PrecF32QP : PrecF32P {
    static constexpr bool framed = true;
    using ST = int8_t;
};

// Read-only typed view of one state buffer: 9 flow planes then 5 thermal
// planes (then, for framed storage, the frame plane t).
template <class T> struct Src {
    const typename T::SF* __restrict__ f;
    const typename T::SG* __restrict__ g;
    const typename FrameStore<T>::type* __restrict__ t;
};
template <class T> struct Dst {
    typename T::SF* __restrict__ f;
    typename T::SG* __restrict__ g;
    typename FrameStore<T>::type* __restrict__ t;
};
template <class T> __host__ __device__ inline Src<T> src_view(const void* base, int plane) {
    Src<T> s;
    s.f = (const typename T::SF*)base;
    s.g = (const typename T::SG*)((const char*)base + (size_t)9 * plane * sizeof(typename T::SF));
    s.t = (const typename FrameStore<T>::type*)(s.g + (size_t)5 * plane);
    return s;
}
template <class T> __host__ __device__ inline Dst<T> dst_view(void* base, int plane) {
    Dst<T> d;
    d.f = (typename T::SF*)base;
    d.g = (typename T::SG*)((char*)base + (size_t)9 * plane * sizeof(typename T::SF));
    d.t = (typename FrameStore<T>::type*)(d.g + (size_t)5 * plane);
    return d;
}
template <class T> __host__ __device__ constexpr size_t buffer_bytes(int plane) {
    return (size_t)plane * (9 * sizeof(typename T::SF) + 5 * sizeof(typename T::SG) +
                            (Framed<T>::value ? sizeof(typename FrameStore<T>::type) : 0));
}

// ---- two nodes in one register pair ------------------------------------------------

// FP32 values of two nodes side by side.  Each +, -, * is one paired FP32
// instruction for both nodes (sm_100-class GPUs), rounded to nearest like its
// scalar counterpart; the pair is never fused into an FMA, so a result may
// differ from the scalar path's (which the compiler contracts) by a rounding.
// Division and sqrt are taken per component.  The type and its functions
// live in a namespace of their own, so that sqrt(float) here keeps meaning
// the CUDA function while sqrt(F2) is found by argument-dependent lookup.
namespace x2 {
struct F2 {
    float2 v;
    F2() = default;
    __device__ __forceinline__ F2(float2 a) : v(a) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit F2(double c) : v(make_float2((float)c, (float)c)) {}
    __device__ __forceinline__ explicit F2(float c) : v(make_float2(c, c)) {}
    __device__ __forceinline__ explicit F2(int c) : v(make_float2((float)c, (float)c)) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
// a - b = a + (-1) b: the product is exact, so this rounds once, as a subtraction does
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.v.x, -a.v.y); }
__device__ __forceinline__ F2 operator/(F2 a, F2 b) { return F2(a.v.x / b.v.x, a.v.y / b.v.y); }
__device__ __forceinline__ F2 operator+(float a, F2 b) { return F2(a) + b; }
__device__ __forceinline__ F2 operator+(F2 a, float b) { return a + F2(b); }
__device__ __forceinline__ F2 operator-(float a, F2 b) { return F2(a) - b; }
__device__ __forceinline__ F2 operator-(F2 a, float b) { return a - F2(b); }
__device__ __forceinline__ F2 operator*(float a, F2 b) { return F2(a) * b; }
__device__ __forceinline__ F2 operator*(F2 a, float b) { return a * F2(b); }
__device__ __forceinline__ F2 sqrt(F2 a) { return F2(sqrtf(a.v.x), sqrtf(a.v.y)); }
__device__ __forceinline__ F2 div_small(F2 a, F2 b) { return F2(__fdividef(a.v.x, b.v.x), __fdividef(a.v.y, b.v.y)); }
}  // namespace x2
using x2::F2;

// a / b for quotients that only scale a small correction (b near 1): the
// fast FP32 division (2 ulp) there, IEEE division in FP64.
__host__ __device__ __forceinline__ double div_small(double a, double b) { return a / b; }
__host__ __device__ __forceinline__ float div_small(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
}

// Sum of the thermal values h (T - T0, or T - T0 - F framed, without the
// source half-step): in the association of n_0 in the increment-form
// collision when INC, else left to right.  Every place that forms a
// temperature from pulled values uses this, so they agree bit for bit.
template <bool INC, class R> __host__ __device__ __forceinline__ R heat_sum(const R (&h)[5]) {
    if constexpr (INC) return ((h[0] + h[1]) + (h[2] + h[3])) + h[4];
    return h[0] + h[1] + h[2] + h[3] + h[4];
}

// x and y momentum of deviations d (m_3 and m_5 of Eq. 9-11), with one
// association of the sums wherever they are taken.
template <class R> __host__ __device__ __forceinline__ R mom_x(const R (&d)[9]) {
    return (d[1] - d[3]) + ((d[5] - d[6]) - (d[7] - d[8]));
}
template <class R> __host__ __device__ __forceinline__ R mom_y(const R (&d)[9]) {
    return (d[2] - d[4]) + ((d[5] + d[6]) - (d[7] + d[8]));
}

// FP16 flow storage: moves each FP32 flow value onto the half-precision grid
// (13 low mantissa bits cleared) with the rounding threshold taken from the
// low mantissa bits of two other populations of the node, instead of
// rounding to nearest.  Those bits change from step to step and do not
// depend on the value rounded, so the rounding error averages out over the
// steps instead of repeating: rounded to nearest, a slowly changing value
// is rounded the same way step after step, and the slow Darcy relaxation
// integrates that bias into the velocity.  The store's conversion to half
// is then exact (in half's normal range; below 2^-14 it rounds once more).
// The threshold is added to the bit pattern, whose low 31 bits are the
// magnitude for either sign.  NaN passes unchanged (infinities stay
// infinite).
__device__ __forceinline__ void dither_to_half(float (&v)[9]) {
    uint32_t b[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) b[i] = __float_as_uint(v[i]);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const uint32_t r = (b[(i + 1) % 9] ^ b[(i + 5) % 9]) & 0x1fffu;
        const float m = __uint_as_float((b[i] + r) & 0xffffe000u);
        v[i] = v[i] != v[i] ? v[i] : m;
    }
}
template <class T> __host__ __device__ constexpr bool half_flow() { return std::is_same<typename T::SF, __half>::value; }

// ---- per-launch coefficients ----------------------------------------------------

// Everything a step needs besides the buffers, in the arithmetic type R.
template <class R> struct Coef {
    R s[9];       // flow relaxation rates (Eq. 20)
    R hs[9];      // 1 - s_k / 2
    R z[5];       // thermal relaxation rates (Eq. 31)
    R hz[5];      // 1 - zeta_k / 2
    R gbeta;      // g beta (buoyancy G = g beta (T - T0) j, Section 2)
    R dTh, dTc;   // wall temperatures minus T0
    R T0;
    R inv_sigma;  // 1 / sigma
    R varpi;      // D2Q5 constant (Eq. 29)
    R inv_csT2;   // 1 / c_sT^2 = 10 / (4 + varpi)
    R wt0, wt1;   // D2Q5 weights w~_0 = (1 - varpi)/5, w~_i = (4 + varpi)/20
    R psi0, psi3; // Psi_0 = Q/sigma, Psi_3 = varpi Q/sigma (Eq. 30)
    R qhalf;      // Q / (2 sigma), the source part of Eq. 36
    R phi;        // uniform porosity
    R c_lin;      // phi nu / K         (uniform porosity)
    R c_quad;     // phi F_phi / sqrt K (uniform porosity)
    R a_lin;      // per-cell: phi nu / K      = a_lin  (1 - phi)^2 / phi^2
    R a_quad;     // per-cell: phi F_phi / sqrt K = a_quad (1 - phi) / phi^2
    R fq, ifq;    // 8-bit temperature frames: quantum (a power of two) and its inverse
    R wt1fq;      // w~_1 fq (exact: fq is a power of two)
};

// Geometry of one lattice in one pair of buffers.
struct Geom {
    int nx, ny;
    int pitch;        // elements per row
    int plane;        // elements per population plane (pitch * ny)
    int thermal_bc;   // 0 side-heated, 1 cooled
    int adi_order;    // 1 or 2
#ifdef LBM_BOUNDS_CHECK
    int* oob;         // counter of accesses outside their plane (bounds-checked build)
#endif
};

// Bounds-checked build (LBM_BOUNDS_CHECK): every population, frame and
// porosity access of the step's pull, wall rule and stores is checked against
// its plane [0, plane) first; an access outside it is skipped (a load reads 0)
// and counted in *gm.oob.  In the normal build the check is compiled away.
__device__ __forceinline__ bool in_plane(const Geom& gm, int o, int n = 1) {
#ifdef LBM_BOUNDS_CHECK
    if (o >= 0 && o <= gm.plane - n) return true;
    atomicAdd(gm.oob, 1);
    return false;
#else
    (void)gm, (void)o, (void)n;
    return true;
#endif
}

// Porosity-dependent drag coefficients (Eq. 4 and Eq. 5 per cell).
template <class R> struct Drag {
    R phi, iphi, c_lin, c_quad;
};

// Drag coefficients of one cell from its porosity (FIELD) or the uniform ones.
template <class R, bool FIELD>
__device__ __forceinline__ Drag<R> drag_of(const Coef<R>& c, R phi) {
    Drag<R> dr;
    if constexpr (FIELD) {
        R iphi = R(1) / phi;
        R om = R(1) - phi;
        R ip2 = iphi * iphi;
        dr.phi = phi;
        dr.iphi = iphi;
        dr.c_lin = c.a_lin * om * om * ip2;
        dr.c_quad = c.a_quad * om * ip2;
    } else {
        dr.phi = c.phi;
        dr.iphi = R(1) / c.phi;
        dr.c_lin = c.c_lin;
        dr.c_quad = c.c_quad;
    }
    return dr;
}

template <class R, bool FIELD, class P>
__device__ __forceinline__ Drag<R> drag_at(const Coef<R>& c, const P* phi_field, int off) {
    if constexpr (FIELD) return drag_of<R, true>(c, Conv<P, R>::ld(phi_field + off));
    return drag_of<R, false>(c, R(0));
}
template <class R, bool FIELD, class P>
__device__ __forceinline__ Drag<R> drag_at(const Coef<R>& c, const Geom& gm, const P* phi_field, int off) {
    if constexpr (FIELD) return drag_at<R, FIELD, P>(c, phi_field, in_plane(gm, off) ? off : 0);
    return drag_of<R, false>(c, R(0));
}

// ---- temperature frames -------------------------------------------------------------

// Frame values as stored (FP32) or as 8-bit integers k with F = k fq.
template <class T, class R>
__device__ __forceinline__ R frame_ld(const Coef<R>& c, const typename FrameStore<T>::type* p) {
    if constexpr (sizeof(typename FrameStore<T>::type) == 1) {
        const int8_t k = T::cg ? __ldca((const signed char*)p) : __ldg((const signed char*)p);
        return R((int)k) * c.fq;
    } else {
        return Conv<typename FrameStore<T>::type, R, T::cg>::ld(p);
    }
}

// The frame a node takes for temperature deviation v, as it will read back,
// and its stored form.
template <class T, class R>
__device__ __forceinline__ R frame_make(const Coef<R>& c, R v, typename FrameStore<T>::type& code) {
    if constexpr (sizeof(typename FrameStore<T>::type) == 1) {
        // a NaN or an overflowing value saturates (the divergence flag reports it)
        const float k = fminf(fmaxf(rintf((float)(v * c.ifq)), -128.f), 127.f);
        code = (typename FrameStore<T>::type)(int)k;
        return R(k) * c.fq;
    } else {
        code = v;
        return v;
    }
}

// The stored code k of an 8-bit frame (F = k fq), and of a node pair.
template <class T>
__device__ __forceinline__ int frame_code(const typename FrameStore<T>::type* p) {
    return (int)(T::cg ? __ldca((const signed char*)p) : __ldg((const signed char*)p));
}
template <class T>
__device__ __forceinline__ char2 frame_pair_code(const typename FrameStore<T>::type* p) {
    return T::cg ? __ldca((const char2*)p) : __ldg((const char2*)p);
}

// Frames of the node pair (x0, x0 + 1), x0 even.
template <class T, class R>
__device__ __forceinline__ void frame_ld2(const Coef<R>& c, const typename FrameStore<T>::type* p, R& a, R& b) {
    if constexpr (sizeof(typename FrameStore<T>::type) == 1) {
        const char2 k = T::cg ? __ldca((const char2*)p) : __ldg((const char2*)p);
        a = R((int)(signed char)k.x) * c.fq;
        b = R((int)(signed char)k.y) * c.fq;
    } else {
        const auto v = Conv2<typename FrameStore<T>::type, R, T::cg>::ld(p);
        a = v.x;
        b = v.y;
    }
}
template <class T>
__device__ __forceinline__ void frame_st2(typename FrameStore<T>::type* p, typename FrameStore<T>::type a,
                                          typename FrameStore<T>::type b) {
    if constexpr (sizeof(typename FrameStore<T>::type) == 1)
        *(char2*)p = make_char2((char)a, (char)b);
    else
        Conv2<typename FrameStore<T>::type, typename FrameStore<T>::type, T::cg>::st(p, a, b);
}

// ---- pull of one node ------------------------------------------------------------

// f_i(x, t+1) = f_i^+(x - e_i, t) (Eq. 18) and g_j likewise (Eq. 35).
// off = y * pitch + x of the receiving node.
template <class T>
__device__ __forceinline__ void pull(const Src<T>& src, const Geom& gm, int off,
                                     typename T::R (&d)[9], typename T::R (&h)[5]) {
    using R = typename T::R;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int o = off - ey9(i) * gm.pitch - ex9(i);
        d[i] = in_plane(gm, o) ? Conv<typename T::SF, R, T::cg>::ld(src.f + i * gm.plane + o) : R(0);
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int o = off - ey9(j) * gm.pitch - ex9(j);
        h[j] = in_plane(gm, o) ? Conv<typename T::SG, R, T::cg>::ld(src.g + j * gm.plane + o) : R(0);
    }
}

template <class T>
__device__ __forceinline__ typename T::R pull_heat(const Src<T>& src, const Geom& gm, int off) {
    using R = typename T::R;
    R t = 0;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int o = off - ey9(j) * gm.pitch - ex9(j);
        t += in_plane(gm, o) ? Conv<typename T::SG, R, T::cg>::ld(src.g + j * gm.plane + o) : R(0);
    }
    return t;
}

// The pull of the node pair off0, off0 + 1 (x0 even): populations with
// e_x = 0 come as one aligned pair access, the others (shifted by one node)
// as two single accesses.
template <class T>
__device__ __forceinline__ void pull_x2(const Src<T>& src, const Geom& gm, int off0, typename T::R (&d0)[9],
                                        typename T::R (&h0)[5], typename T::R (&d1)[9], typename T::R (&h1)[5]) {
    using R = typename T::R;
    using SF = typename T::SF;
    using SG = typename T::SG;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int o = off0 - ey9(i) * gm.pitch - ex9(i);
        const SF* p = src.f + i * gm.plane + o;
        if (ex9(i) == 0) {
            const auto v = in_plane(gm, o, 2) ? Conv2<SF, R, T::cg>::ld(p) : decltype(Conv2<SF, R, T::cg>::ld(p)){};
            d0[i] = v.x;
            d1[i] = v.y;
        } else {
            d0[i] = in_plane(gm, o) ? Conv<SF, R, T::cg>::ld(p) : R(0);
            d1[i] = in_plane(gm, o + 1) ? Conv<SF, R, T::cg>::ld(p + 1) : R(0);
        }
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int o = off0 - ey9(j) * gm.pitch - ex9(j);
        const SG* p = src.g + j * gm.plane + o;
        if (ex9(j) == 0) {
            const auto v = in_plane(gm, o, 2) ? Conv2<SG, R, T::cg>::ld(p) : decltype(Conv2<SG, R, T::cg>::ld(p)){};
            h0[j] = v.x;
            h1[j] = v.y;
        } else {
            h0[j] = in_plane(gm, o) ? Conv<SG, R, T::cg>::ld(p) : R(0);
            h1[j] = in_plane(gm, o + 1) ? Conv<SG, R, T::cg>::ld(p + 1) : R(0);
        }
    }
}

// frame_in for the node pair off0, off0 + 1 (x0 even): the pair's own frames
// and those of the rows above and below come as pairs, the east and west
// neighbours' as single values.
template <class T>
__device__ __forceinline__ void frame_in_x2(const Coef<typename T::R>& c, const Src<T>& src, const Geom& gm,
                                            int off0, typename T::R (&h0)[5], typename T::R (&h1)[5],
                                            typename T::R& F0, typename T::R& F1) {
    using R = typename T::R;
    if constexpr (sizeof(typename FrameStore<T>::type) == 1) {
        // 8-bit frames: differences taken on the integers, as in frame_in
        char2 own = make_char2(0, 0), sth = own, nth = own;
        signed char w = 0, e = 0;
        if (in_plane(gm, off0, 2)) own = frame_pair_code<T>(src.t + off0);
        if (in_plane(gm, off0 - gm.pitch, 2)) sth = frame_pair_code<T>(src.t + off0 - gm.pitch);  // j = 2: y - 1
        if (in_plane(gm, off0 + gm.pitch, 2)) nth = frame_pair_code<T>(src.t + off0 + gm.pitch);  // j = 4: y + 1
        if (in_plane(gm, off0 - 1)) w = (signed char)frame_code<T>(src.t + off0 - 1);
        if (in_plane(gm, off0 + 2)) e = (signed char)frame_code<T>(src.t + off0 + 2);
        const int k0 = (signed char)own.x, k1 = (signed char)own.y;
        h0[1] += c.wt1fq * R((int)w - k0);
        h1[1] += c.wt1fq * R(k0 - k1);
        h0[2] += c.wt1fq * R((int)(signed char)sth.x - k0);
        h1[2] += c.wt1fq * R((int)(signed char)sth.y - k1);
        h0[3] += c.wt1fq * R(k1 - k0);
        h1[3] += c.wt1fq * R((int)e - k1);
        h0[4] += c.wt1fq * R((int)(signed char)nth.x - k0);
        h1[4] += c.wt1fq * R((int)(signed char)nth.y - k1);
        F0 = R(k0) * c.fq;
        F1 = R(k1) * c.fq;
    } else {
        R n0 = R(0), n1 = R(0), s0 = R(0), s1 = R(0), w = R(0), e = R(0);
        F0 = F1 = R(0);
        if (in_plane(gm, off0, 2)) frame_ld2<T>(c, src.t + off0, F0, F1);
        if (in_plane(gm, off0 - gm.pitch, 2)) frame_ld2<T>(c, src.t + off0 - gm.pitch, s0, s1);  // j = 2: y - 1
        if (in_plane(gm, off0 + gm.pitch, 2)) frame_ld2<T>(c, src.t + off0 + gm.pitch, n0, n1);  // j = 4: y + 1
        if (in_plane(gm, off0 - 1)) w = frame_ld<T>(c, src.t + off0 - 1);
        if (in_plane(gm, off0 + 2)) e = frame_ld<T>(c, src.t + off0 + 2);
        h0[1] += c.wt1 * (w - F0);
        h1[1] += c.wt1 * (F0 - F1);
        h0[2] += c.wt1 * (s0 - F0);
        h1[2] += c.wt1 * (s1 - F1);
        h0[3] += c.wt1 * (F1 - F0);
        h1[3] += c.wt1 * (e - F1);
        h0[4] += c.wt1 * (n0 - F0);
        h1[4] += c.wt1 * (n1 - F1);
    }
}

// Framed storage: thermal values pulled into node off were stored in the
// frames of the nodes they came from; re-express them in this node's frame F
// (add w~_j (F(x - e_j) - F), j >= 1: nearby frames subtract exactly) and
// return F.
template <class T>
__device__ __forceinline__ typename T::R frame_in(const Coef<typename T::R>& c, const Src<T>& src, const Geom& gm,
                                                  int off, typename T::R (&h)[5]) {
    using R = typename T::R;
    if constexpr (sizeof(typename FrameStore<T>::type) == 1) {
        // 8-bit frames: w~_1 (F_s - F) = (w~_1 fq) (k_s - k), the same rounding, the
        // difference taken on the integers
        const int k = in_plane(gm, off) ? frame_code<T>(src.t + off) : 0;
#pragma unroll
        for (int j = 1; j < 5; ++j) {
            const int o = off - ey9(j) * gm.pitch - ex9(j);
            h[j] += c.wt1fq * R((in_plane(gm, o) ? frame_code<T>(src.t + o) : 0) - k);
        }
        return R(k) * c.fq;
    } else {
        const R F = in_plane(gm, off) ? frame_ld<T>(c, src.t + off) : R(0);
#pragma unroll
        for (int j = 1; j < 5; ++j) {
            const int o = off - ey9(j) * gm.pitch - ex9(j);
            h[j] += c.wt1 * ((in_plane(gm, o) ? frame_ld<T>(c, src.t + o) : R(0)) - F);
        }
        return F;
    }
}

// T - T0 - F(x) at node off from the pulled thermal values (framed storage), and F(x).
template <class T>
__device__ __forceinline__ typename T::R pull_heat_framed(const Coef<typename T::R>& c, const Src<T>& src,
                                                          const Geom& gm, int off, typename T::R& F) {
    using R = typename T::R;
    R h[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int o = off - ey9(j) * gm.pitch - ex9(j);
        h[j] = in_plane(gm, o) ? Conv<typename T::SG, R, T::cg>::ld(src.g + j * gm.plane + o) : R(0);
    }
    F = frame_in<T>(c, src, gm, off, h);
    return heat_sum<IncForm<T>::value>(h);
}

// ---- macroscopic values -------------------------------------------------------------

template <class R> struct Macro {
    R ux, uy;  // velocity (Eq. 21)
    R dux, duy;  // u - j, j = (m_3, m_5) of the populations the collision starts from
    R dP;      // phi p - rho0 c_s^2 (Eq. 23)
    R dT;      // T - T0 (Eq. 36)
    R Fx, Fy;  // total force (Eq. 4)
    R umag;    // |u|
    R F, dTl;  // framed storage: the node's frame and T - T0 - F (else 0 and dT)
};

// Eq. 36, Section 2 buoyancy, Eq. 22, Eq. 21, Eq. 23, Eq. 4 at a fluid node.
// CR: type of the coefficients (R, or float for the node pair F2).  FR: the
// thermal values h are relative to the frame F (framed storage).
template <class R, class CR, bool FR = false, bool INC = false>
__device__ __forceinline__ Macro<R> fluid_macros(const Coef<CR>& c, const Drag<R>& dr,
                                                 const R (&d)[9], const R (&h)[5], R F = R(0)) {
    Macro<R> m;
    // n_0 of the thermal collision (INC: summed in its association)
    const R n0 = heat_sum<INC>(h);
    if constexpr (FR) {
        m.F = F;
        m.dTl = n0 + c.qhalf;
        m.dT = F + m.dTl;
    } else {
        m.dT = n0 + c.qhalf;
        m.dTl = m.dT;
    }
    const R Gy = c.gbeta * m.dT;
    const R jx = INC ? mom_x(d) : (d[1] - d[3]) + (d[5] - d[6]) - (d[7] - d[8]);
    const R jy = INC ? mom_y(d) : (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
    const R by = R(0.5) * dr.phi * Gy;  // half the buoyancy impulse
    const R vx = jx;
    const R vy = jy + by;
    // Eq. 22, u = v / (l0 + sqrt(l0^2 + l1 |v|)) with l0 = 1/2 + c_lin/4, written
    // as u = v - v g / (1 + g), g = l0 + sqrt(l0^2 + l1 |v|) - 1 (of the order
    // of the drag per step): the collision adds u - j to the momentum, and
    // that difference is formed here from small terms only, so its rounding
    // scales with g and not with |u|.  (Formed as u - j from a rounded u, the
    // error would be a fixed fraction of u per step, which the slow Darcy
    // relaxation integrates into a velocity error of order 1e-7 / drag.)
    // The direct form without INC (FP64 and FP16-flow storage, see collide).
    const R l1 = R(0.5) * dr.c_quad;
    const R vm = sqrt(vx * vx + vy * vy);
    if constexpr (INC) {
        const R cc = R(0.25) * dr.c_lin;
        const R e = cc + cc * cc + l1 * vm;  // l0^2 + l1 |v| - 1/4
        const R g = cc + div_small(e, sqrt(R(0.25) + e) + R(0.5));
        const R den = div_small(R(1), R(1) + g);
        const R gd = g * den;
        m.dux = -(vx * gd);
        m.duy = by - vy * gd;
        m.ux = jx + m.dux;
        m.uy = jy + m.duy;
        m.umag = vm * den;
    } else {
        const R l0 = R(0.5) + R(0.25) * dr.c_lin;
        const R den = R(1) / (l0 + sqrt(l0 * l0 + l1 * vm));
        m.ux = vx * den;
        m.uy = vy * den;
        m.umag = vm * den;
        m.dux = m.ux - jx;
        m.duy = m.uy - jy;
    }
    const R uu = m.ux * m.ux + m.uy * m.uy;
    const R s18 = (d[1] + d[2] + d[3] + d[4]) + (d[5] + d[6] + d[7] + d[8]);
    // c_s^2 / (1 - w_0) = 3/5 and rho0 s_0(u) = -(2/3) |u|^2 / phi
    m.dP = R(0.6) * s18 - R(0.4) * uu * dr.iphi;
    const R drag = dr.c_lin + dr.c_quad * m.umag;
    m.Fx = -drag * m.ux;
    m.Fy = -drag * m.uy + dr.phi * Gy;
    return m;
}

// ---- collision ------------------------------------------------------------------------

// Eq. 17 with m_eq of Eq. 16 and S of Eq. 19, then f+ = M^-1 m+ (Eq. 18,
// M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4));
// Eq. 34 with n_eq of Eq. 29 and Psi of Eq. 30, then g+ = N^-1 n+ (Eq. 35,
// N^-1 = N^T diag(1/5, 1/2, 1/2, 1/20, 1/4)).  In place on d and h, as
// increments: f+ = f + M^-1 (m+ - m), g+ = g + N^-1 (n+ - n).  Equal in exact
// arithmetic; in FP32 the rounded factors 1/9, 1/6, 1/36, 1/5 ... then scale
// the change of a step instead of the whole moment, where 6 fl(1/6) != 1
// would bias the momentum by 3e-8 of itself every step (a velocity error
// of 3e-8 / drag once the Darcy relaxation has integrated it).  INC = false
// forms f+ = M^-1 m+ from the new moments instead (the same in exact
// arithmetic; fewer live registers): FP64, whose rounding is far below
// that bias, and FP16-flow storage, whose rounding is far above it.
template <class R, class CR, bool FR = false, bool INC = false>
__host__ __device__ __forceinline__ void collide(const Coef<CR>& c, R iphi, const Macro<R>& mc, R (&d)[9],
                                        R (&h)[5]) {
    // m = M d (Eq. 9-11), as a deviation from the rest moments; m_3 - u_x
    // and m_5 - u_y come with the macroscopic values (mc.dux, mc.duy)
    const R a = (d[1] + d[2]) + (d[3] + d[4]);
    const R b = (d[5] + d[6]) + (d[7] + d[8]);
    const R ex13 = d[1] - d[3], ey24 = d[2] - d[4];
    const R dx = (d[5] - d[6]) - (d[7] - d[8]);  // diagonal x-momentum
    const R dy = (d[5] + d[6]) - (d[7] + d[8]);  // diagonal y-momentum
    const R m0 = d[0] + a + b;
    const R m1 = R(-4) * d[0] - a + R(2) * b;
    const R m2 = R(4) * d[0] - R(2) * a + b;
    const R m4 = R(-2) * ex13 + dx;
    const R m6 = R(-2) * ey24 + dy;
    const R m7 = (d[1] - d[2]) + (d[3] - d[4]);
    const R m8 = (d[5] - d[6]) + (d[7] - d[8]);

    // m_eq (Eq. 16) minus rest moments
    const R ux = mc.ux, uy = mc.uy;
    const R uu = ux * ux + uy * uy;
    const R q = R(3) * uu * iphi;
    const R eq1 = R(6) * mc.dP + q;
    const R eq2 = R(-9) * mc.dP - q;
    const R eq7 = (ux * ux - uy * uy) * iphi;
    const R eq8 = ux * uy * iphi;
    // S (Eq. 19)
    const R uF = ux * mc.Fx + uy * mc.Fy;
    const R S1 = R(6) * uF * iphi;
    const R S7 = R(2) * (ux * mc.Fx - uy * mc.Fy) * iphi;
    const R S8 = (ux * mc.Fy + uy * mc.Fx) * iphi;

    // Eq. 17: m+ - m = -s (m - m_eq) + (1 - s/2) S (INC: that alone, else
    // with m added), scaled by the diagonal of M^-1
    R p0, p1, p2, p3, p4, p5, p6, p7, p8;
    if constexpr (INC) {
        p0 = -(c.s[0] * m0) * R(1.0 / 9.0);
        p1 = (c.hs[1] * S1 - c.s[1] * (m1 - eq1)) * R(1.0 / 36.0);
        p2 = (-(c.hs[2] * S1) - c.s[2] * (m2 - eq2)) * R(1.0 / 36.0);
        p3 = (c.s[3] * mc.dux + c.hs[3] * mc.Fx) * R(1.0 / 6.0);
        p4 = (-(c.hs[4] * mc.Fx) - c.s[4] * (m4 + ux)) * R(1.0 / 12.0);
        p5 = (c.s[5] * mc.duy + c.hs[5] * mc.Fy) * R(1.0 / 6.0);
        p6 = (-(c.hs[6] * mc.Fy) - c.s[6] * (m6 + uy)) * R(1.0 / 12.0);
        p7 = (c.hs[7] * S7 - c.s[7] * (m7 - eq7)) * R(0.25);
        p8 = (c.hs[8] * S8 - c.s[8] * (m8 - eq8)) * R(0.25);
    } else {
        const R m3 = ex13 + dx, m5 = ey24 + dy;
        p0 = (m0 - c.s[0] * m0) * R(1.0 / 9.0);
        p1 = (m1 - c.s[1] * (m1 - eq1) + c.hs[1] * S1) * R(1.0 / 36.0);
        p2 = (m2 - c.s[2] * (m2 - eq2) - c.hs[2] * S1) * R(1.0 / 36.0);
        p3 = (m3 - c.s[3] * (m3 - ux) + c.hs[3] * mc.Fx) * R(1.0 / 6.0);
        p4 = (m4 - c.s[4] * (m4 + ux) - c.hs[4] * mc.Fx) * R(1.0 / 12.0);
        p5 = (m5 - c.s[5] * (m5 - uy) + c.hs[5] * mc.Fy) * R(1.0 / 6.0);
        p6 = (m6 - c.s[6] * (m6 + uy) - c.hs[6] * mc.Fy) * R(1.0 / 12.0);
        p7 = (m7 - c.s[7] * (m7 - eq7) + c.hs[7] * S7) * R(0.25);
        p8 = (m8 - c.s[8] * (m8 - eq8) + c.hs[8] * S8) * R(0.25);
    }

    // f+ = M^T p (columns of Eq. 11)
    const R r1 = p0 - p1 - R(2) * p2;  // common part of the axis directions
    const R r5 = p0 + R(2) * p1 + p2;  // common part of the diagonals
    const R x34 = p3 - R(2) * p4, y56 = p5 - R(2) * p6;
    const R x34d = p3 + p4, y56d = p5 + p6;
    if constexpr (INC) {
        d[0] = d[0] + (p0 - R(4) * p1 + R(4) * p2);
        d[1] = d[1] + (r1 + x34 + p7);
        d[2] = d[2] + (r1 + y56 - p7);
        d[3] = d[3] + (r1 - x34 + p7);
        d[4] = d[4] + (r1 - y56 - p7);
        d[5] = d[5] + (r5 + x34d + y56d + p8);
        d[6] = d[6] + (r5 - x34d + y56d - p8);
        d[7] = d[7] + (r5 - x34d - y56d + p8);
        d[8] = d[8] + (r5 + x34d - y56d - p8);
    } else {
        d[0] = p0 - R(4) * p1 + R(4) * p2;
        d[1] = r1 + x34 + p7;
        d[2] = r1 + y56 - p7;
        d[3] = r1 - x34 + p7;
        d[4] = r1 - y56 - p7;
        d[5] = r5 + x34d + y56d + p8;
        d[6] = r5 - x34d + y56d - p8;
        d[7] = r5 - x34d - y56d + p8;
        d[8] = r5 + x34d - y56d - p8;
    }

    // thermal: n = N h (Eq. 27-28), deviation from T0 (1, 0, 0, varpi, 0)
    const R n0 = INC ? ((h[0] + h[1]) + (h[2] + h[3])) + h[4] : (h[0] + h[1]) + (h[2] + h[3]) + h[4];
    const R n1 = h[1] - h[3];
    const R n2 = h[2] - h[4];
    const R n3 = R(-4) * h[0] + (h[1] + h[2]) + (h[3] + h[4]);
    const R n4 = (h[1] - h[2]) + (h[3] - h[4]);
    const R T = c.T0 + mc.dT;
    const R ne1 = ux * T * c.inv_sigma;
    const R ne2 = uy * T * c.inv_sigma;
    // framed storage: n and the conserved part of n_eq are taken relative to
    // T0 + F, the flux part (u T / sigma) uses the absolute T
    const R dTn = FR ? mc.dTl : mc.dT;
    const R ne3 = c.varpi * dTn;
    if constexpr (INC) {
        // Eq. 34 as n+ - n = -zeta (n - n_eq) + (1 - zeta/2) Psi
        const R q0 = (c.hz[0] * c.psi0 - c.z[0] * (n0 - dTn)) * R(0.2);
        const R q1 = -(c.z[1] * (n1 - ne1)) * R(0.5);
        const R q2 = -(c.z[2] * (n2 - ne2)) * R(0.5);
        const R q3 = (c.hz[3] * c.psi3 - c.z[3] * (n3 - ne3)) * R(0.05);
        const R q4 = -(c.z[4] * n4) * R(0.25);
        h[0] = h[0] + (q0 - R(4) * q3);
        h[1] = h[1] + (q0 + q1 + q3 + q4);
        h[2] = h[2] + (q0 + q2 + q3 - q4);
        h[3] = h[3] + (q0 - q1 + q3 + q4);
        h[4] = h[4] + (q0 - q2 + q3 - q4);
    } else {
        const R q0 = (n0 - c.z[0] * (n0 - dTn) + c.hz[0] * c.psi0) * R(0.2);
        const R q1 = (n1 - c.z[1] * (n1 - ne1)) * R(0.5);
        const R q2 = (n2 - c.z[2] * (n2 - ne2)) * R(0.5);
        const R q3 = (n3 - c.z[3] * (n3 - ne3) + c.hz[3] * c.psi3) * R(0.05);
        const R q4 = (n4 - c.z[4] * n4) * R(0.25);
        h[0] = q0 - R(4) * q3;
        h[1] = q0 + q1 + q3 + q4;
        h[2] = q0 + q2 + q3 - q4;
        h[3] = q0 - q1 + q3 + q4;
        h[4] = q0 - q2 + q3 - q4;
    }
}

// ---- wall rule ----------------------------------------------------------------------------

// Inward normal of a node: (0, 0) for fluid nodes, the diagonal at corners.
struct Normal {
    int dx, dy;
};
__device__ __forceinline__ Normal normal_of(const Geom& gm, int x, int y) {
    Normal n;
    n.dx = (x == 0) ? 1 : (x == gm.nx - 1 ? -1 : 0);
    n.dy = (y == 0) ? 1 : (y == gm.ny - 1 ? -1 : 0);
    return n;
}

// Non-equilibrium extrapolation (Section 4, ref. [43]) at wall node (x, y)
// with inward normal nr: reads the pulled populations of the inner neighbour
// x_f = x + nr (and of x + 2 nr for the second-order adiabatic variant),
// writes the wall node's populations into d, h and returns the imposed
// macroscopic values (u = 0, p_b = p_f, T_b; force phi_b G(T_b) j).
template <class T, bool FIELD>
__device__ __forceinline__ Macro<typename T::R> wall_node(const Coef<typename T::R>& c, const Geom& gm,
                                                          const Src<T>& src, const typename T::P* phi_field,
                                                          int x, int y, Normal nr,
                                                          const Drag<typename T::R>& drb,
                                                          typename T::R (&d)[9], typename T::R (&h)[5]) {
    using R = typename T::R;
    constexpr bool FR = Framed<T>::value;
    const int offf = (y + nr.dy) * gm.pitch + (x + nr.dx);
    R df[9], hf[5];
    pull<T>(src, gm, offf, df, hf);
    R Ff = R(0), Fb = R(0);  // frames of the inner neighbour and of this wall node
    if constexpr (FR) {
        Ff = frame_in<T>(c, src, gm, offf, hf);
        Fb = in_plane(gm, y * gm.pitch + x) ? frame_ld<T>(c, src.t + y * gm.pitch + x) : R(0);
    }
    const Drag<R> drf = drag_at<R, FIELD, typename T::P>(c, gm, phi_field, offf);
    const Macro<R> mf = fluid_macros<R, R, FR, IncForm<T>::value>(c, drf, df, hf, Ff);

    Macro<R> mb;
    mb.ux = R(0);
    mb.uy = R(0);
    mb.umag = R(0);
    // p_b = p_f:  P_b = phi_b p_f, P = rho0 c_s^2 + dP
    if constexpr (FIELD) {
        mb.dP = (drb.phi * drf.iphi) * (R(1.0 / 3.0) + mf.dP) - R(1.0 / 3.0);
    } else {
        mb.dP = mf.dP;
    }
    const bool dirichlet = (gm.thermal_bc == 1) || (nr.dx != 0);
    if constexpr (FR) {
        // the wall temperature relative to this node's frame, from differences of nearby frames
        mb.F = Fb;
        if (dirichlet) {
            mb.dTl = ((gm.thermal_bc == 1) ? c.dTc : (x == 0 ? c.dTh : c.dTc)) - Fb;
        } else if (gm.adi_order == 2) {
            const int offff = (y + 2 * nr.dy) * gm.pitch + (x + 2 * nr.dx);
            R Fff;
            const R dTlff = pull_heat_framed<T>(c, src, gm, offff, Fff) + c.qhalf;
            mb.dTl = (R(4) * ((Ff - Fb) + mf.dTl) - ((Fff - Fb) + dTlff)) * R(1.0 / 3.0);
        } else {
            mb.dTl = (Ff - Fb) + mf.dTl;
        }
        mb.dT = Fb + mb.dTl;
    } else {
        if (dirichlet) {
            mb.dT = (gm.thermal_bc == 1) ? c.dTc : (x == 0 ? c.dTh : c.dTc);
        } else if (gm.adi_order == 2) {
            const int offff = (y + 2 * nr.dy) * gm.pitch + (x + 2 * nr.dx);
            const R dTff = pull_heat<T>(src, gm, offff) + c.qhalf;
            mb.dT = (R(4) * mf.dT - dTff) * R(1.0 / 3.0);
        } else {
            mb.dT = mf.dT;
        }
    }
    mb.Fx = R(0);
    mb.Fy = drb.phi * c.gbeta * mb.dT;

    // f_b = f_eq(P_b, 0) + f_f - f_eq(P_f, u_f) (Eq. 13-14 as deviations):
    // f_eq,i - w_i rho0 = 3 w_i dP + s_i(u) (i >= 1), -(5/3) dP + s_0(u) (i = 0)
    const R ddP = mb.dP - mf.dP;
    const R ux = mf.ux, uy = mf.uy;
    const R uu = ux * ux + uy * uy;
    const R ip = drf.iphi;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const R eu = R(ex9(i)) * ux + R(ey9(i)) * uy;
        const R si = R(w9(i)) * (R(3) * eu + R(4.5) * eu * eu * ip - R(1.5) * uu * ip);
        const R cP = (i == 0) ? R(-5.0 / 3.0) : R(3.0 * w9(i));
        d[i] = df[i] - si + cP * ddP;
    }
    mb.dux = -mom_x(d);  // u_b = 0
    mb.duy = -mom_y(d);
    // g_b = g_eq(T_b, 0) + g_f - g_eq(T_f, u_f) (Eq. 37, first occurrence); framed:
    // T_b - T_f from the frames' difference and the local parts, the result
    // re-expressed in this node's frame
    const R Tf = c.T0 + mf.dT;
    // (framed: w~ (T_b - T_f) + w~ (F_f - F_b) = w~ (dTl_b - dTl_f))
    const R ddT = FR ? mb.dTl - mf.dTl : mb.dT - mf.dT;
    const R adv = Tf * c.inv_sigma * c.inv_csT2 * c.wt1;
    const R sh0 = c.wt0 * ddT;
    const R sh1 = c.wt1 * ddT;
    h[0] = hf[0] + sh0;
    h[1] = hf[1] + sh1 - adv * ux;
    h[2] = hf[2] + sh1 - adv * uy;
    h[3] = hf[3] + sh1 + adv * ux;
    h[4] = hf[4] + sh1 + adv * uy;
    return mb;
}

// Post-stream state of node (x, y) (pull + wall rule) and its macroscopic values.
template <class T, bool FIELD>
__device__ __forceinline__ Macro<typename T::R> node_state(const Coef<typename T::R>& c, const Geom& gm,
                                                           const Src<T>& src, const typename T::P* phi_field,
                                                           int x, int y, Drag<typename T::R>& dr,
                                                           typename T::R (&d)[9], typename T::R (&h)[5]) {
    using R = typename T::R;
    const int off = y * gm.pitch + x;
    dr = drag_at<R, FIELD, typename T::P>(c, gm, phi_field, off);
    const Normal nr = normal_of(gm, x, y);
    if (nr.dx == 0 && nr.dy == 0) {
        pull<T>(src, gm, off, d, h);
        if constexpr (Framed<T>::value) {
            const R F = frame_in<T>(c, src, gm, off, h);
            return fluid_macros<R, R, true, IncForm<T>::value>(c, dr, d, h, F);
        }
        return fluid_macros<R, R, false, IncForm<T>::value>(c, dr, d, h);
    }
    return wall_node<T, FIELD>(c, gm, src, phi_field, x, y, nr, dr, d, h);
}

// Framed storage: re-expresses the collided thermal values, relative to the
// frame mc.F they were computed in, in the node's new frame (T - T0 in the
// frame's storage type) and stores that frame.
template <class T>
__device__ __forceinline__ void frame_out(const Coef<typename T::R>& c, const Geom& gm, const Dst<T>& dst, int off,
                                          const Macro<typename T::R>& mc, typename T::R (&h)[5]) {
    using R = typename T::R;
    typename FrameStore<T>::type code;
    const R Fn = frame_make<T>(c, mc.dT, code);  // F + dTl as the frame stores it: the new frame
    const R shift = Fn - mc.F;                    // exact: both are frame values
    h[0] -= c.wt0 * shift;
#pragma unroll
    for (int j = 1; j < 5; ++j) h[j] -= c.wt1 * shift;
    if (in_plane(gm, off)) dst.t[off] = code;
}

// ---- wall-column temperatures -------------------------------------------------------

// The Nusselt number (Eq. 38) reads T at the five node columns next to each
// vertical wall.  An observing step stores T - T0 of those nodes of the
// post-stream state as it computes them: obs[kObsCols y + k] holds node
// x = k (k < 5) and node x = nx - 1 - (k - 5) (k >= 5), in FP64, the value
// node_dT reports for a node off the walls (framed storage: frame and local
// part added in FP64).  A node of a narrow lattice may fill two slots.
constexpr int kObsCols = 10;

__device__ __forceinline__ void obs_put(const Geom& gm, double* obs, int x, int y, double v) {
    if (x < 5) obs[kObsCols * y + x] = v;
    if (x >= gm.nx - 5) obs[kObsCols * y + 5 + (gm.nx - 1 - x)] = v;
}

template <class T>
__device__ __forceinline__ double obs_value(const Macro<typename T::R>& m) {
    if constexpr (Framed<T>::value)
        return (double)m.F + (double)m.dTl;
    else
        return (double)m.dT;
}

// One node of the step: pull (or wall rule), collide, store; OBS: also the
// node's temperature into obs when it lies in a wall column.  That store
// comes after all arithmetic: a branch between the macroscopic values and
// the collision would change where the compiler fuses multiply-adds, and
// with it the rounding of the lattice.
template <class T, bool FIELD, bool OBS = false>
__device__ __forceinline__ void update_node(const Coef<typename T::R>& c, const Geom& gm, const Src<T>& src,
                                            const Dst<T>& dst, const typename T::P* phi, int x, int y,
                                            int* status, double* obs = nullptr) {
    using R = typename T::R;
    R d[9], h[5];
    Drag<R> dr;
    const Macro<R> mc = node_state<T, FIELD>(c, gm, src, phi, x, y, dr, d, h);
    if (!(mc.umag < R(0.5))) atomicOr(status, 1);  // also catches NaN
    collide<R, R, Framed<T>::value, IncForm<T>::value>(c, dr.iphi, mc, d, h);
    if constexpr (half_flow<T>()) dither_to_half(d);
    const int off = y * gm.pitch + x;
    if constexpr (Framed<T>::value) frame_out<T>(c, gm, dst, off, mc, h);
    if (in_plane(gm, off)) {
#pragma unroll
        for (int i = 0; i < 9; ++i) Conv<typename T::SF, R, T::cg>::st(dst.f + i * gm.plane + off, d[i]);
#pragma unroll
        for (int j = 0; j < 5; ++j) Conv<typename T::SG, R, T::cg>::st(dst.g + j * gm.plane + off, h[j]);
    }
    if constexpr (OBS) obs_put(gm, obs, x, y, obs_value<T>(mc));
}

// Two fluid nodes from their pulled values in one pass of F2 arithmetic (FP32
// arithmetic types only): about half the arithmetic instructions of two nodes.
// Framed storage: the frames F0, F1 the pulled thermal values b0, b1 are
// relative to (frame_in), and the frame change of both nodes on the way out.
// VEC: the nodes are x-neighbours off1 = off0 + 1 with x0 even, stored as
// pairs.
template <class T, bool OBS = false, bool VEC = false>
__device__ __forceinline__ void collide_fluid_pair_x2(const Coef<float>& c, const Geom& gm, const Dst<T>& dst,
                                                      const float (&a0)[9], const float (&b0)[5],
                                                      const float (&a1)[9], const float (&b1)[5],
                                                      const Drag<float>& r0, const Drag<float>& r1, int off0,
                                                      int off1, int* status, int x0 = 0, int y0 = 0, int x1 = 0,
                                                      int y1 = 0, double* obs = nullptr, float F0 = 0.f,
                                                      float F1 = 0.f) {
    constexpr bool FR = Framed<T>::value;
    Drag<F2> dr;
    dr.phi = F2(r0.phi, r1.phi);
    dr.iphi = F2(r0.iphi, r1.iphi);
    dr.c_lin = F2(r0.c_lin, r1.c_lin);
    dr.c_quad = F2(r0.c_quad, r1.c_quad);
    F2 d[9], h[5];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = F2(a0[i], a1[i]);
#pragma unroll
    for (int j = 0; j < 5; ++j) h[j] = F2(b0[j], b1[j]);
    const Macro<F2> m = fluid_macros<F2, float, FR>(c, dr, d, h, F2(F0, F1));
    if (!(m.umag.v.x < 0.5f) || !(m.umag.v.y < 0.5f)) atomicOr(status, 1);
    collide<F2, float, FR>(c, dr.iphi, m, d, h);
    if constexpr (half_flow<T>()) {
        float v0[9], v1[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            v0[i] = d[i].v.x;
            v1[i] = d[i].v.y;
        }
        dither_to_half(v0);
        dither_to_half(v1);
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = F2(v0[i], v1[i]);
    }
    if constexpr (FR) {
        typename FrameStore<T>::type k0, k1;
        const float s0 = frame_make<T>(c, m.dT.v.x, k0) - m.F.v.x;  // exact: frame values
        const float s1 = frame_make<T>(c, m.dT.v.y, k1) - m.F.v.y;
        const F2 sh(s0, s1);
        h[0] = h[0] - c.wt0 * sh;
#pragma unroll
        for (int j = 1; j < 5; ++j) h[j] = h[j] - c.wt1 * sh;
        if constexpr (VEC) {
            if (in_plane(gm, off0, 2)) frame_st2<T>(dst.t + off0, k0, k1);
        } else {
            if (in_plane(gm, off0)) dst.t[off0] = k0;
            if (in_plane(gm, off1)) dst.t[off1] = k1;
        }
    }
    if constexpr (VEC) {
        if (in_plane(gm, off0, 2)) {
#pragma unroll
            for (int i = 0; i < 9; ++i)
                Conv2<typename T::SF, float, T::cg>::st(dst.f + i * gm.plane + off0, d[i].v.x, d[i].v.y);
#pragma unroll
            for (int j = 0; j < 5; ++j)
                Conv2<typename T::SG, float, T::cg>::st(dst.g + j * gm.plane + off0, h[j].v.x, h[j].v.y);
        }
    } else {
        if (in_plane(gm, off0)) {
#pragma unroll
            for (int i = 0; i < 9; ++i) Conv<typename T::SF, float, T::cg>::st(dst.f + i * gm.plane + off0, d[i].v.x);
#pragma unroll
            for (int j = 0; j < 5; ++j) Conv<typename T::SG, float, T::cg>::st(dst.g + j * gm.plane + off0, h[j].v.x);
        }
        if (in_plane(gm, off1)) {
#pragma unroll
            for (int i = 0; i < 9; ++i) Conv<typename T::SF, float, T::cg>::st(dst.f + i * gm.plane + off1, d[i].v.y);
#pragma unroll
            for (int j = 0; j < 5; ++j) Conv<typename T::SG, float, T::cg>::st(dst.g + j * gm.plane + off1, h[j].v.y);
        }
    }
    if constexpr (OBS) {
        // lane-wise IEEE sums: the same values as the scalar path
        if constexpr (FR) {
            obs_put(gm, obs, x0, y0, (double)m.F.v.x + (double)m.dTl.v.x);
            obs_put(gm, obs, x1, y1, (double)m.F.v.y + (double)m.dTl.v.y);
        } else {
            obs_put(gm, obs, x0, y0, (double)m.dT.v.x);
            obs_put(gm, obs, x1, y1, (double)m.dT.v.y);
        }
    }
}

template <class T, bool FIELD, bool OBS = false>
__device__ __forceinline__ void update_fluid_pair_x2(const Coef<float>& c, const Geom& gm, const Src<T>& src,
                                                     const Dst<T>& dst, const typename T::P* phi, int x0, int y0,
                                                     int x1, int y1, int* status, double* obs = nullptr) {
    const int off0 = y0 * gm.pitch + x0, off1 = y1 * gm.pitch + x1;
    float a0[9], b0[5], a1[9], b1[5];
    pull<T>(src, gm, off0, a0, b0);
    pull<T>(src, gm, off1, a1, b1);
    float F0 = 0.f, F1 = 0.f;
    if constexpr (Framed<T>::value) {
        F0 = frame_in<T>(c, src, gm, off0, b0);
        F1 = frame_in<T>(c, src, gm, off1, b1);
    }
    const Drag<float> r0 = drag_at<float, FIELD, typename T::P>(c, gm, phi, off0);
    const Drag<float> r1 = drag_at<float, FIELD, typename T::P>(c, gm, phi, off1);
    collide_fluid_pair_x2<T, OBS>(c, gm, dst, a0, b0, a1, b1, r0, r1, off0, off1, status, x0, y0, x1, y1, obs, F0,
                                  F1);
}

// Two nodes at once: when both are fluid nodes all 28 loads are issued before
// any arithmetic (twice the bytes in flight of one node per thread); nodes
// outside the lattice (valid = false) or on walls take the one-node path.
template <class T, bool FIELD, bool OBS = false>
__device__ __forceinline__ void update_pair(const Coef<typename T::R>& c, const Geom& gm, const Src<T>& src,
                                            const Dst<T>& dst, const typename T::P* phi, int x0, int y0,
                                            bool v0, int x1, int y1, bool v1, int* status, double* obs = nullptr) {
    using R = typename T::R;
    const bool f0 = v0 && x0 > 0 && x0 < gm.nx - 1 && y0 > 0 && y0 < gm.ny - 1;
    const bool f1 = v1 && x1 > 0 && x1 < gm.nx - 1 && y1 > 0 && y1 < gm.ny - 1;
    if constexpr (Paired<T>::value) {
        if (f0 && f1) {
            update_fluid_pair_x2<T, FIELD, OBS>(c, gm, src, dst, phi, x0, y0, x1, y1, status, obs);
            return;
        }
    }
    if (f0 && f1) {
        R d0[9], h0[5], d1[9], h1[5];
        const int off0 = y0 * gm.pitch + x0, off1 = y1 * gm.pitch + x1;
        constexpr bool FR = Framed<T>::value;
        pull<T>(src, gm, off0, d0, h0);
        pull<T>(src, gm, off1, d1, h1);
        R F0 = R(0), F1 = R(0);
        if constexpr (FR) {
            F0 = frame_in<T>(c, src, gm, off0, h0);
            F1 = frame_in<T>(c, src, gm, off1, h1);
        }
        const Drag<R> dr0 = drag_at<R, FIELD, typename T::P>(c, gm, phi, off0);
        const Drag<R> dr1 = drag_at<R, FIELD, typename T::P>(c, gm, phi, off1);
        const Macro<R> m0 = fluid_macros<R, R, FR, IncForm<T>::value>(c, dr0, d0, h0, F0);
        const Macro<R> m1 = fluid_macros<R, R, FR, IncForm<T>::value>(c, dr1, d1, h1, F1);
        if (!(m0.umag < R(0.5)) || !(m1.umag < R(0.5))) atomicOr(status, 1);
        collide<R, R, FR, IncForm<T>::value>(c, dr0.iphi, m0, d0, h0);
        collide<R, R, FR, IncForm<T>::value>(c, dr1.iphi, m1, d1, h1);
        if constexpr (FR) {
            frame_out<T>(c, gm, dst, off0, m0, h0);
            frame_out<T>(c, gm, dst, off1, m1, h1);
        }
        if (in_plane(gm, off0) && in_plane(gm, off1)) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                Conv<typename T::SF, R, T::cg>::st(dst.f + i * gm.plane + off0, d0[i]);
                Conv<typename T::SF, R, T::cg>::st(dst.f + i * gm.plane + off1, d1[i]);
            }
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                Conv<typename T::SG, R, T::cg>::st(dst.g + j * gm.plane + off0, h0[j]);
                Conv<typename T::SG, R, T::cg>::st(dst.g + j * gm.plane + off1, h1[j]);
            }
        }
        if constexpr (OBS) {
            obs_put(gm, obs, x0, y0, obs_value<T>(m0));
            obs_put(gm, obs, x1, y1, obs_value<T>(m1));
        }
        return;
    }
    if (v0) update_node<T, FIELD, OBS>(c, gm, src, dst, phi, x0, y0, status, obs);
    if (v1) update_node<T, FIELD, OBS>(c, gm, src, dst, phi, x1, y1, status, obs);
}

// Two nodes side by side, (x0, y) and (x0 + 1, y) with x0 even: when both are
// fluid nodes the populations with e_x = 0, the stores and the frames move
// as aligned pairs (about a third fewer memory instructions than two nodes
// apart); otherwise each valid node takes the one-node path.
template <class T, bool FIELD, bool OBS = false>
__device__ __forceinline__ void update_xpair(const Coef<typename T::R>& c, const Geom& gm, const Src<T>& src,
                                             const Dst<T>& dst, const typename T::P* phi, int x0, int y,
                                             int* status, double* obs = nullptr) {
    using R = typename T::R;
    constexpr bool FR = Framed<T>::value;
    const int x1 = x0 + 1;
    if (x0 > 0 && x1 < gm.nx - 1 && y > 0 && y < gm.ny - 1) {
        const int off0 = y * gm.pitch + x0, off1 = off0 + 1;
        R d0[9], h0[5], d1[9], h1[5];
        pull_x2<T>(src, gm, off0, d0, h0, d1, h1);
        R F0 = R(0), F1 = R(0);
        if constexpr (FR) frame_in_x2<T>(c, src, gm, off0, h0, h1, F0, F1);
        const Drag<R> dr0 = drag_at<R, FIELD, typename T::P>(c, gm, phi, off0);
        const Drag<R> dr1 = drag_at<R, FIELD, typename T::P>(c, gm, phi, off1);
        if constexpr (Paired<T>::value) {
            collide_fluid_pair_x2<T, OBS, true>(c, gm, dst, d0, h0, d1, h1, dr0, dr1, off0, off1, status, x0, y, x1,
                                                y, obs, F0, F1);
        } else {
            const Macro<R> m0 = fluid_macros<R, R, FR, IncForm<T>::value>(c, dr0, d0, h0, F0);
            const Macro<R> m1 = fluid_macros<R, R, FR, IncForm<T>::value>(c, dr1, d1, h1, F1);
            if (!(m0.umag < R(0.5)) || !(m1.umag < R(0.5))) atomicOr(status, 1);
            collide<R, R, FR, IncForm<T>::value>(c, dr0.iphi, m0, d0, h0);
            collide<R, R, FR, IncForm<T>::value>(c, dr1.iphi, m1, d1, h1);
            if constexpr (FR) {
                typename FrameStore<T>::type k0, k1;
                const R s0 = frame_make<T>(c, m0.dT, k0) - m0.F;  // exact: frame values
                const R s1 = frame_make<T>(c, m1.dT, k1) - m1.F;
                h0[0] -= c.wt0 * s0;
                h1[0] -= c.wt0 * s1;
#pragma unroll
                for (int j = 1; j < 5; ++j) {
                    h0[j] -= c.wt1 * s0;
                    h1[j] -= c.wt1 * s1;
                }
                if (in_plane(gm, off0, 2)) frame_st2<T>(dst.t + off0, k0, k1);
            }
            if (in_plane(gm, off0, 2)) {
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    Conv2<typename T::SF, R, T::cg>::st(dst.f + i * gm.plane + off0, d0[i], d1[i]);
#pragma unroll
                for (int j = 0; j < 5; ++j)
                    Conv2<typename T::SG, R, T::cg>::st(dst.g + j * gm.plane + off0, h0[j], h1[j]);
            }
            if constexpr (OBS) {
                obs_put(gm, obs, x0, y, obs_value<T>(m0));
                obs_put(gm, obs, x1, y, obs_value<T>(m1));
            }
        }
        return;
    }
    if (x0 < gm.nx) update_node<T, FIELD, OBS>(c, gm, src, dst, phi, x0, y, status, obs);
    if (x1 < gm.nx) update_node<T, FIELD, OBS>(c, gm, src, dst, phi, x1, y, status, obs);
}

// T - T0 of the post-stream state at node (x, y), pulled from B_{n-1}
// (the wall rule's temperature on wall nodes), in FP64 (framed storage adds
// the frame to the local part in FP64, so the value keeps its precision).
template <class T>
__device__ __forceinline__ double node_dT(const Coef<typename T::R>& c, const Geom& gm, const Src<T>& prev, int x,
                                          int y) {
    using R = typename T::R;
    const Normal nr = normal_of(gm, x, y);
    if constexpr (Framed<T>::value) {
        R F;
        if (nr.dx == 0 && nr.dy == 0) {
            const R l = pull_heat_framed<T>(c, prev, gm, y * gm.pitch + x, F) + c.qhalf;
            return (double)F + (double)l;
        }
        if (gm.thermal_bc == 1) return (double)c.dTc;
        if (nr.dx != 0) return (double)(x == 0 ? c.dTh : c.dTc);
        const R lf = pull_heat_framed<T>(c, prev, gm, (y + nr.dy) * gm.pitch + x, F) + c.qhalf;
        if (gm.adi_order == 2) {
            R Fff;
            const R lff = pull_heat_framed<T>(c, prev, gm, (y + 2 * nr.dy) * gm.pitch + x, Fff) + c.qhalf;
            return (4.0 * ((double)F + (double)lf) - ((double)Fff + (double)lff)) / 3.0;
        }
        return (double)F + (double)lf;
    } else {
        if (nr.dx == 0 && nr.dy == 0) return (double)(pull_heat<T>(prev, gm, y * gm.pitch + x) + c.qhalf);
        if (gm.thermal_bc == 1) return (double)c.dTc;
        if (nr.dx != 0) return (double)(x == 0 ? c.dTh : c.dTc);
        const R dTf = pull_heat<T>(prev, gm, (y + nr.dy) * gm.pitch + x) + c.qhalf;
        if (gm.adi_order == 2) {
            const R dTff = pull_heat<T>(prev, gm, (y + 2 * nr.dy) * gm.pitch + x) + c.qhalf;
            return (double)((R(4) * dTf - dTff) * R(1.0 / 3.0));
        }
        return (double)dTf;
    }
}

// node_dT of node (x, y), x = k (k < 5) or nx - 1 - (k - 5), from the wall
// columns an observing step stored (obs_put): the stored value off the walls;
// on the walls the wall rule's temperature, imposed on the vertical walls and,
// on the adiabatic rows, taken from the stored rows next to them in the
// arithmetic node_dT uses, so both give the same bits.
template <class T>
__device__ __forceinline__ double obs_dT(const Coef<typename T::R>& c, const Geom& gm, const double* obs, int k,
                                         int y) {
    using R = typename T::R;
    const int x = k < 5 ? k : gm.nx - 1 - (k - 5);
    const Normal nr = normal_of(gm, x, y);
    if (nr.dx == 0 && nr.dy == 0) return obs[kObsCols * y + k];
    if (gm.thermal_bc == 1) return (double)c.dTc;
    if (nr.dx != 0) return (double)(x == 0 ? c.dTh : c.dTc);
    const double tf = obs[kObsCols * (y + nr.dy) + k];
    if (gm.adi_order == 2) {
        const double tff = obs[kObsCols * (y + 2 * nr.dy) + k];
        if constexpr (Framed<T>::value)
            return (4.0 * tf - tff) / 3.0;
        else
            return (double)((R(4) * R(tf) - R(tff)) * R(1.0 / 3.0));
    }
    return tf;
}

// The larger of a and b, NaN when either is NaN (fmax would drop it, and a
// maximum over a lattice holding NaN would look finite).
__device__ __forceinline__ double fmax_nan(double a, double b) { return (a > b || a != a) ? a : b; }

// Block-wide reduction of four doubles: max, max, sum, sum (result in thread
// 0); the maxima keep NaN.
__device__ __forceinline__ void block_reduce4(double v[4], double* sh /* 4 * 32 */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v[0] = fmax_nan(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
        v[1] = fmax_nan(v[1], __shfl_xor_sync(0xffffffffu, v[1], o));
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
            v[0] = fmax_nan(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
            v[1] = fmax_nan(v[1], __shfl_xor_sync(0xffffffffu, v[1], o));
            v[2] += __shfl_xor_sync(0xffffffffu, v[2], o);
            v[3] += __shfl_xor_sync(0xffffffffu, v[3], o);
        }
    }
}

// Mean Nusselt numbers (Eq. 38) of both vertical walls over the whole block
// (valid in thread 0): Nu(y) = -L dT/dx / dT with the one-sided five-point
// derivative (-25 T0 + 48 T1 - 36 T2 + 16 T3 - 3 T4) / 12, trapezoidal mean
// over y, FP64.  sh: 4 * 32 doubles of shared memory.
template <class T>
__device__ __forceinline__ void nusselt_block(const Coef<typename T::R>& c, const Geom& gm, const Src<T>& prev,
                                              double L, double dT, double* sh, double* nu_hot, double* nu_cold) {
    double w[4] = {0.0, 0.0, 0.0, 0.0};
    const int nx = gm.nx;
    for (int y = threadIdx.x; y < gm.ny; y += blockDim.x) {
        double tl[5], tr[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            tl[k] = (double)node_dT<T>(c, gm, prev, k, y);
            tr[k] = (double)node_dT<T>(c, gm, prev, nx - 1 - k, y);
        }
        const double dl = (-25.0 * tl[0] + 48.0 * tl[1] - 36.0 * tl[2] + 16.0 * tl[3] - 3.0 * tl[4]) / 12.0;
        const double dr = (25.0 * tr[0] - 48.0 * tr[1] + 36.0 * tr[2] - 16.0 * tr[3] + 3.0 * tr[4]) / 12.0;
        const double wt = (y == 0 || y == gm.ny - 1) ? 0.5 : 1.0;
        w[2] += wt * (-L * dl / dT);
        w[3] += wt * (-L * dr / dT);
    }
    block_reduce4(w, sh);
    *nu_hot = w[2] / (double)(gm.ny - 1);
    *nu_cold = w[3] / (double)(gm.ny - 1);
}

}  // namespace lbm
