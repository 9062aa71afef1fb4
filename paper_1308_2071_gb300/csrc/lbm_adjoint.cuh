// Reverse mode of one node of the fused step, for the discrete adjoint.
//
// The forward map of one node (pull, wall rule, collision; Sections 3-4) is
// differentiated by hand: given the adjoint of the node's post-collision
// populations (lambda), these functions return the adjoint of the pulled
// populations it read and of the porosity it used.  Porosity enters through
// the per-cell Ergun drag (Eq. 4-5) and the equilibria (Eq. 14, 16, 19, 23).
// All functions are plain arithmetic (host and device) so that they can be
// checked against finite differences of the forward functions.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// Forward intermediates of the macroscopic values at a fluid node (Eq. 4, 5,
// 21-23, 36), with the per-cell drag coefficients.
template <class R> struct Tape {
    R phi, iphi, om, ip2, c_lin, c_quad;
    R dT, Gy, vx, vy, l0, l1, vm, q, den, ux, uy, um, uu, dP, drag, Fx, Fy;
};

template <class R>
__host__ __device__ inline void tape_node(const Coef<R>& c, R phi, const R (&d)[9], const R (&h)[5], Tape<R>& t) {
    t.phi = phi;
    t.iphi = R(1) / phi;
    t.om = R(1) - phi;
    t.ip2 = t.iphi * t.iphi;
    t.c_lin = c.a_lin * t.om * t.om * t.ip2;
    t.c_quad = c.a_quad * t.om * t.ip2;
    t.dT = (h[0] + h[1] + h[2] + h[3] + h[4]) + c.qhalf;
    t.Gy = c.gbeta * t.dT;
    const R jx = (d[1] - d[3]) + (d[5] - d[6]) - (d[7] - d[8]);
    const R jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
    t.vx = jx;
    t.vy = jy + R(0.5) * t.phi * t.Gy;
    t.l0 = R(0.5) + R(0.25) * t.c_lin;
    t.l1 = R(0.5) * t.c_quad;
    t.vm = sqrt(t.vx * t.vx + t.vy * t.vy);
    t.q = sqrt(t.l0 * t.l0 + t.l1 * t.vm);
    t.den = R(1) / (t.l0 + t.q);
    t.ux = t.vx * t.den;
    t.uy = t.vy * t.den;
    t.um = t.vm * t.den;
    t.uu = t.ux * t.ux + t.uy * t.uy;
    const R s18 = (d[1] + d[2] + d[3] + d[4]) + (d[5] + d[6] + d[7] + d[8]);
    t.dP = R(0.6) * s18 - R(0.4) * t.uu * t.iphi;
    t.drag = t.c_lin + t.c_quad * t.um;
    t.Fx = -t.drag * t.ux;
    t.Fy = -t.drag * t.uy + t.phi * t.Gy;
}

// Adjoint seeds of the macroscopic values.
template <class R> struct MacroBar {
    R ux, uy, um, dP, dT, Fx, Fy, iphi, phi;
};

// m = M x (rows of Eq. 11); used both for moments and for M lambda.
template <class R> __host__ __device__ inline void apply_M(const R (&x)[9], R (&m)[9]) {
    const R a = (x[1] + x[2]) + (x[3] + x[4]);
    const R b = (x[5] + x[6]) + (x[7] + x[8]);
    const R ex13 = x[1] - x[3], ey24 = x[2] - x[4];
    const R dx = (x[5] - x[6]) - (x[7] - x[8]);
    const R dy = (x[5] + x[6]) - (x[7] + x[8]);
    m[0] = x[0] + a + b;
    m[1] = R(-4) * x[0] - a + R(2) * b;
    m[2] = R(4) * x[0] - R(2) * a + b;
    m[3] = ex13 + dx;
    m[4] = R(-2) * ex13 + dx;
    m[5] = ey24 + dy;
    m[6] = R(-2) * ey24 + dy;
    m[7] = (x[1] - x[2]) + (x[3] - x[4]);
    m[8] = (x[5] - x[6]) + (x[7] - x[8]);
}

// y = M^T p (columns of Eq. 11).
template <class R> __host__ __device__ inline void apply_MT(const R (&p)[9], R (&y)[9]) {
    const R r1 = p[0] - p[1] - R(2) * p[2];
    const R r5 = p[0] + R(2) * p[1] + p[2];
    const R x34 = p[3] - R(2) * p[4], y56 = p[5] - R(2) * p[6];
    const R x34d = p[3] + p[4], y56d = p[5] + p[6];
    y[0] = p[0] - R(4) * p[1] + R(4) * p[2];
    y[1] = r1 + x34 + p[7];
    y[2] = r1 + y56 - p[7];
    y[3] = r1 - x34 + p[7];
    y[4] = r1 - y56 - p[7];
    y[5] = r5 + x34d + y56d + p[8];
    y[6] = r5 - x34d + y56d - p[8];
    y[7] = r5 - x34d - y56d + p[8];
    y[8] = r5 + x34d - y56d - p[8];
}

template <class R> __host__ __device__ inline void apply_N(const R (&x)[5], R (&n)[5]) {
    n[0] = (x[0] + x[1]) + (x[2] + x[3]) + x[4];
    n[1] = x[1] - x[3];
    n[2] = x[2] - x[4];
    n[3] = R(-4) * x[0] + (x[1] + x[2]) + (x[3] + x[4]);
    n[4] = (x[1] - x[2]) + (x[3] - x[4]);
}

template <class R> __host__ __device__ inline void apply_NT(const R (&q)[5], R (&y)[5]) {
    y[0] = q[0] - R(4) * q[3];
    y[1] = q[0] + q[1] + q[3] + q[4];
    y[2] = q[0] + q[2] + q[3] - q[4];
    y[3] = q[0] - q[1] + q[3] + q[4];
    y[4] = q[0] - q[2] + q[3] - q[4];
}

// Reverse of the collision (Eq. 17 with Eq. 16 and 19; Eq. 34 with Eq. 29) at
// a node with macroscopic values (ux, uy, dP, dT, Fx, Fy, 1/phi).  Writes the
// adjoint of the pre-collision populations through the moments into db, hb
// and returns the seeds of the macroscopic values.  With moving = false the
// velocity is an imposed constant (wall nodes) and gets no seed.
template <class R>
__host__ __device__ inline MacroBar<R> collide_adjoint(const Coef<R>& c, R ux, R uy, R dT, R Fx, R Fy, R iphi,
                                                       const R (&lf)[9], const R (&lh)[5], R (&db)[9],
                                                       R (&hb)[5]) {
    const R rm[9] = {R(1.0 / 9.0), R(1.0 / 36.0), R(1.0 / 36.0), R(1.0 / 6.0), R(1.0 / 12.0),
                     R(1.0 / 6.0), R(1.0 / 12.0), R(0.25),       R(0.25)};
    R pb[9], mb[9], eqb[9], Sb[9];
    apply_M(lf, pb);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const R a = pb[k] * rm[k];
        mb[k] = a * (R(1) - c.s[k]);
        eqb[k] = a * c.s[k];
        Sb[k] = a * c.hs[k];
    }
    apply_MT(mb, db);

    MacroBar<R> bar;
    const R uu = ux * ux + uy * uy;
    bar.dP = R(6) * eqb[1] - R(9) * eqb[2];
    R uu_b = R(3) * iphi * (eqb[1] - eqb[2]);
    bar.iphi = R(3) * uu * (eqb[1] - eqb[2]) + (ux * ux - uy * uy) * eqb[7] + ux * uy * eqb[8];
    bar.ux = eqb[3] - eqb[4] + R(2) * ux * iphi * eqb[7] + uy * iphi * eqb[8];
    bar.uy = eqb[5] - eqb[6] - R(2) * uy * iphi * eqb[7] + ux * iphi * eqb[8];
    // forcing moments (S_2 = -S_1, S_4 = -S_3, S_6 = -S_5)
    const R uF = ux * Fx + uy * Fy;
    const R S1b = Sb[1] - Sb[2];
    const R uF_b = R(6) * iphi * S1b;
    bar.iphi += R(6) * uF * S1b + R(2) * (ux * Fx - uy * Fy) * Sb[7] + (ux * Fy + uy * Fx) * Sb[8];
    bar.Fx = Sb[3] - Sb[4] + R(2) * ux * iphi * Sb[7] + uy * iphi * Sb[8];
    bar.Fy = Sb[5] - Sb[6] - R(2) * uy * iphi * Sb[7] + ux * iphi * Sb[8];
    bar.ux += R(2) * Fx * iphi * Sb[7] + Fy * iphi * Sb[8];
    bar.uy += R(-2) * Fy * iphi * Sb[7] + Fx * iphi * Sb[8];
    bar.ux += Fx * uF_b;
    bar.uy += Fy * uF_b;
    bar.Fx += ux * uF_b;
    bar.Fy += uy * uF_b;
    bar.ux += R(2) * ux * uu_b;
    bar.uy += R(2) * uy * uu_b;

    // thermal
    const R rn[5] = {R(0.2), R(0.5), R(0.5), R(0.05), R(0.25)};
    R qb[5], nb[5], neb[5];
    apply_N(lh, qb);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const R a = qb[k] * rn[k];
        nb[k] = a * (R(1) - c.z[k]);
        neb[k] = a * c.z[k];
    }
    apply_NT(nb, hb);
    const R T = c.T0 + dT;
    bar.dT = neb[0] + c.varpi * neb[3] + (ux * neb[1] + uy * neb[2]) * c.inv_sigma;
    bar.ux += T * c.inv_sigma * neb[1];
    bar.uy += T * c.inv_sigma * neb[2];
    bar.um = R(0);
    bar.phi = R(0);
    return bar;
}

// Reverse of tape_node: adds the adjoint of the pulled populations and of the
// porosity for the seeds in bar.
template <class R>
__host__ __device__ inline void macro_adjoint(const Coef<R>& c, const Tape<R>& t, const MacroBar<R>& bar,
                                              R (&db)[9], R (&hb)[5], R& phib) {
    // F = -drag u + phi G j (Eq. 4)
    const R drag_b = -t.ux * bar.Fx - t.uy * bar.Fy;
    R ux_b = bar.ux - t.drag * bar.Fx;
    R uy_b = bar.uy - t.drag * bar.Fy;
    R phi_b = bar.phi + t.Gy * bar.Fy;
    R Gy_b = t.phi * bar.Fy;
    R clin_b = drag_b;
    R cquad_b = t.um * drag_b;
    R um_b = bar.um + t.c_quad * drag_b;
    // dP = 0.6 s18 - 0.4 uu / phi (Eq. 23)
    const R s18_b = R(0.6) * bar.dP;
    const R uu_b = R(-0.4) * t.iphi * bar.dP;
    R iphi_b = bar.iphi - R(0.4) * t.uu * bar.dP;
    ux_b += R(2) * t.ux * uu_b;
    uy_b += R(2) * t.uy * uu_b;
    // u = v den, |u| = |v| den (Eq. 21)
    R vx_b = t.den * ux_b;
    R vy_b = t.den * uy_b;
    R vm_b = t.den * um_b;
    const R den_b = t.vx * ux_b + t.vy * uy_b + t.vm * um_b;
    const R D_b = -t.den * t.den * den_b;
    R l0_b = D_b;
    const R q_b = D_b;
    const R arg_b = t.q > R(0) ? q_b / (R(2) * t.q) : R(0);
    l0_b += R(2) * t.l0 * arg_b;
    const R l1_b = t.vm * arg_b;
    vm_b += t.l1 * arg_b;
    // |v| has no derivative at v = 0; the Forchheimer term's is taken as 0 there
    if (t.vm > R(0)) {
        vx_b += t.vx / t.vm * vm_b;
        vy_b += t.vy / t.vm * vm_b;
    }
    clin_b += R(0.25) * l0_b;
    cquad_b += R(0.5) * l1_b;
    // v = j + phi G / 2 (Eq. 22), G = g beta (T - T0)
    phi_b += R(0.5) * t.Gy * vy_b;
    Gy_b += R(0.5) * t.phi * vy_b;
    const R dT_b = bar.dT + c.gbeta * Gy_b;
    const R jx_b = vx_b, jy_b = vy_b;
#pragma unroll
    for (int i = 1; i < 9; ++i) db[i] += s18_b;
    db[1] += jx_b;
    db[3] -= jx_b;
    db[2] += jy_b;
    db[4] -= jy_b;
    db[5] += jx_b + jy_b;
    db[6] += -jx_b + jy_b;
    db[7] += -jx_b - jy_b;
    db[8] += jx_b - jy_b;
#pragma unroll
    for (int j = 0; j < 5; ++j) hb[j] += dT_b;
    // Ergun drag per cell (Eq. 5): c_lin = a_lin (1-phi)^2 / phi^2, c_quad = a_quad (1-phi) / phi^2
    const R om_b = c.a_lin * R(2) * t.om * t.ip2 * clin_b + c.a_quad * t.ip2 * cquad_b;
    const R ip2_b = c.a_lin * t.om * t.om * clin_b + c.a_quad * t.om * cquad_b;
    iphi_b += R(2) * t.iphi * ip2_b;
    phi_b += -t.iphi * t.iphi * iphi_b - om_b;
    phib += phi_b;
}

// Reverse of a fluid node: lambda of its post-collision populations ->
// adjoint of its pulled populations (db, hb) and of its porosity.
template <class R>
__host__ __device__ inline void fluid_node_adjoint(const Coef<R>& c, const Tape<R>& t, const R (&lf)[9],
                                                   const R (&lh)[5], R (&db)[9], R (&hb)[5], R& phib) {
    MacroBar<R> bar = collide_adjoint<R>(c, t.ux, t.uy, t.dT, t.Fx, t.Fy, t.iphi, lf, lh, db, hb);
    macro_adjoint<R>(c, t, bar, db, hb, phib);
}

// Reverse of a wall node (first-order adiabatic walls): its post-collision
// populations depend on the pulled populations of its inner neighbour x_f
// (tape tf), on phi_b and on phi_f.  Adds to dfb, hfb (adjoint of x_f's pulled
// populations) and to phib_f; returns the adjoint of phi_b.
template <class R>
__host__ __device__ inline R wall_node_adjoint(const Coef<R>& c, const Tape<R>& tf, R phi_b, bool dirichlet,
                                               R dT_wall, const R (&lf)[9], const R (&lh)[5], R (&dfb)[9],
                                               R (&hfb)[5], R& phib_f) {
    // forward imposed values: P_b = phi_b p_f, T_b, u = 0, F = phi_b g beta dT_b j
    const R dPb = phi_b * tf.iphi * (R(1.0 / 3.0) + tf.dP) - R(1.0 / 3.0);
    const R dTb = dirichlet ? dT_wall : tf.dT;
    const R Fyb = phi_b * c.gbeta * dTb;
    R db_wall[9], hb_wall[5];
    MacroBar<R> wb = collide_adjoint<R>(c, R(0), R(0), dTb, R(0), Fyb, R(1) / phi_b, lf, lh, db_wall, hb_wall);
    R dPb_b = wb.dP;
    R dTb_b = wb.dT;
    // F_y = phi_b g beta dT_b (the velocity is imposed, so its seeds are dropped)
    R phib_b = c.gbeta * dTb * wb.Fy;
    dTb_b += phi_b * c.gbeta * wb.Fy;

    // wall populations: d_b = d_f - s(u_f; phi_f) + cP (dP_b - dP_f)
    MacroBar<R> fb = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    R cPsum = R(0);
    R uu_b = R(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        dfb[i] += db_wall[i];
        const R cP = (i == 0) ? R(-5.0 / 3.0) : R(3.0 * w9(i));
        cPsum += cP * db_wall[i];
        const R sb = -db_wall[i];
        const R eu = R(ex9(i)) * tf.ux + R(ey9(i)) * tf.uy;
        const R w = R(w9(i));
        const R eu_b = sb * w * (R(3) + R(9) * eu * tf.iphi);
        fb.ux += R(ex9(i)) * eu_b;
        fb.uy += R(ey9(i)) * eu_b;
        uu_b += sb * w * R(-1.5) * tf.iphi;
        fb.iphi += sb * w * (R(4.5) * eu * eu - R(1.5) * tf.uu);
    }
    fb.ux += R(2) * tf.ux * uu_b;
    fb.uy += R(2) * tf.uy * uu_b;
    dPb_b += cPsum;
    fb.dP -= cPsum;
    // thermal wall populations: h_b = h_f + w~ (dT_b - dT_f) -+ adv u_f
    const R adv = (c.T0 + tf.dT) * c.inv_sigma * c.inv_csT2 * c.wt1;
#pragma unroll
    for (int j = 0; j < 5; ++j) hfb[j] += hb_wall[j];
    const R ddT_b = c.wt0 * hb_wall[0] + c.wt1 * ((hb_wall[1] + hb_wall[2]) + (hb_wall[3] + hb_wall[4]));
    const R adv_b = -tf.ux * hb_wall[1] - tf.uy * hb_wall[2] + tf.ux * hb_wall[3] + tf.uy * hb_wall[4];
    fb.ux += adv * (hb_wall[3] - hb_wall[1]);
    fb.uy += adv * (hb_wall[4] - hb_wall[2]);
    dTb_b += ddT_b;
    fb.dT -= ddT_b;
    fb.dT += c.inv_sigma * c.inv_csT2 * c.wt1 * adv_b;
    if (!dirichlet) fb.dT += dTb_b;
    // P_b = phi_b (rho0 c_s^2 + dP_f) / phi_f
    phib_b += tf.iphi * (R(1.0 / 3.0) + tf.dP) * dPb_b;
    fb.iphi += phi_b * (R(1.0 / 3.0) + tf.dP) * dPb_b;
    fb.dP += phi_b * tf.iphi * dPb_b;
    macro_adjoint<R>(c, tf, fb, dfb, hfb, phib_f);
    return phib_b;
}

// Forward of a wall node built from the same formulas as wall_node (for the
// finite-difference checks of wall_node_adjoint).
template <class R>
__host__ __device__ inline void wall_node_forward(const Coef<R>& c, const Tape<R>& tf, const R (&df)[9],
                                                  const R (&hf)[5], R phi_b, bool dirichlet, R dT_wall,
                                                  R (&d)[9], R (&h)[5]) {
    Macro<R> mb;
    mb.ux = R(0);
    mb.uy = R(0);
    mb.umag = R(0);
    mb.dP = phi_b * tf.iphi * (R(1.0 / 3.0) + tf.dP) - R(1.0 / 3.0);
    mb.dT = dirichlet ? dT_wall : tf.dT;
    mb.Fx = R(0);
    mb.Fy = phi_b * c.gbeta * mb.dT;
    const R ddP = mb.dP - tf.dP;
    const R uu = tf.uu;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const R eu = R(ex9(i)) * tf.ux + R(ey9(i)) * tf.uy;
        const R si = R(w9(i)) * (R(3) * eu + R(4.5) * eu * eu * tf.iphi - R(1.5) * uu * tf.iphi);
        const R cP = (i == 0) ? R(-5.0 / 3.0) : R(3.0 * w9(i));
        d[i] = df[i] - si + cP * ddP;
    }
    mb.dux = -mom_x(d);
    mb.duy = -mom_y(d);
    const R ddT = mb.dT - tf.dT;
    const R adv = (c.T0 + tf.dT) * c.inv_sigma * c.inv_csT2 * c.wt1;
    h[0] = hf[0] + c.wt0 * ddT;
    h[1] = hf[1] + c.wt1 * ddT - adv * tf.ux;
    h[2] = hf[2] + c.wt1 * ddT - adv * tf.uy;
    h[3] = hf[3] + c.wt1 * ddT + adv * tf.ux;
    h[4] = hf[4] + c.wt1 * ddT + adv * tf.uy;
    collide<R>(c, R(1) / phi_b, mb, d, h);
}

// Forward of a fluid node from its pulled populations (for the checks).
template <class R>
__host__ __device__ inline void fluid_node_forward(const Coef<R>& c, R phi, R (&d)[9], R (&h)[5]) {
    Tape<R> t;
    tape_node<R>(c, phi, d, h, t);
    Macro<R> m;
    m.ux = t.ux;
    m.uy = t.uy;
    m.umag = t.um;
    m.dP = t.dP;
    m.dT = t.dT;
    m.Fx = t.Fx;
    m.Fy = t.Fy;
    m.dux = t.ux - mom_x(d);
    m.duy = t.uy - mom_y(d);
    collide<R>(c, t.iphi, m, d, h);
}

}  // namespace lbm
