// sde_transport.cu -- persistent transport kernel of the jump-SDE proton
// engine (arXiv 2511.03115, Sec. 2.1.2, Eq. VSDE) and its small companions
// (spot preparation, single-step probe, dose conversion).
//
// Execution model: one proton history per lane.  Warps are persistent: a warp
// claims a batch of history ids from a global cursor, hands them to its idle
// lanes, and advances all live lanes one Euler-Maruyama step per iteration.
// By default a warp refills only when all 32 lanes are idle (ballot + popc
// ranks), so it carries a cohort of histories of one spot in lock-step.  The
// per-step physics comes from FP32 tables read through L1 (optionally staged
// in shared memory); each step draws one Philox4x32-10 block keyed by (seed,
// history, step); a large-angle event is sampled at the top of the next
// iteration, outside the step body; the energy lost in the step is committed as a 64-bit
// fixed-point integer atomic, so the tally does not depend on execution order.
#include <math.h>

#include "sde_internal.cuh"
#include "sde_transport.h"

namespace sde {

// Per-unit-density step quantities at one energy (see the hot-row layout in
// sde_internal.cuh): c = varsigma_1 Delta, s = sqrt(varsigma_2^2 Delta),
// w = Lynch-Dahl w, tg = t / g(w) (Brownian time over g), sj = jump rate x Delta,
// sn = its non-elastic part; k, f = table interval and fraction.
struct Phys {
    float c, s, w, tg, sj, sn, f;
    int k;
};

__device__ __forceinline__ void grid_pos(const KParams& P, float E, int& k, float& f) {
    float xf = (__log2f(E) - P.lg2_emin) * P.inv_dlg2;
    xf = fminf(fmaxf(xf, 0.f), (float)(P.N - 1));
    k = min((int)xf, P.N - 2);
    f = xf - (float)k;
}

__device__ __forceinline__ Phys lookup(const float4* tab, const KParams& P, int m, float E) {
    int k;
    float f;
    grid_pos(P, E, k, f);
    // at most 16 materials x 4096 points x 3 rows: a 32-bit offset
    const float4* r = tab + (uint32_t)(m * P.N + k) * (uint32_t)kRowFloat4;
    float4 a = r[0], b = r[1], c = r[2];
    const float mp = (float)kProtonMass;
    float tot = E + mp;
    float rp2 = __fdividef(1.f, E * (E + 2.f * mp));  // 1/p^2
    float ib2 = tot * tot * rp2;                      // 1/beta^2
    float rE = __fdividef(1.f, E);
    Phys ph;
    ph.c = fmaf(a.y, f, a.x) * ib2;
    ph.s = fmaf(a.w, f, a.z);
    ph.w = c.z * fmaf(b.y, f, b.x) * ib2;
    ph.tg = c.w * ib2 * rp2;
    ph.sn = fmaf(c.y, f, c.x);
    ph.sj = fmaf(fmaf(b.w, f, b.z), rE * rE, ph.sn);
    ph.k = k;
    ph.f = f;
    return ph;
}

// Primitive of the hydrogen (Mott) Coulomb law in the forward variable s = 1 - mu:
// G = 2 mu/(1-mu^2) - sin(eta ln((1+mu)/(1-mu)))/(2 eta).
__device__ __forceinline__ float mott_prim(float s, float eta) {
    float L = __logf((2.f - s) / s);
    return __fdividef(2.f * (1.f - s), s * (2.f - s)) - __fdividef(__sinf(eta * L), 2.f * eta);
}

// 1 - cos(theta_c) of the variable cut-off theta_c^2 = th2 (clamped to [1e-4, 1] rad as the
// oracle does); a series below theta_c^2 = 0.01, where 1 - cosf would lose digits.
__device__ __forceinline__ float cut_s(float th2) {
    th2 = fminf(fmaxf(th2, 1e-8f), 1.f);
    if (th2 < 0.01f) return 0.5f * th2 * (1.f - th2 * (1.f / 12.f) * (1.f - th2 * (1.f / 30.f)));
    return 1.f - cosf(sqrtf(th2));
}

// Large-angle elastic rate x Delta per unit density at cut-off s_c (Sec. 2.1.3, Eq.
// large_elastic_cm and its hydrogen form): R (1/s_c - 1/2) + Hc G(s_c) - Hc G(mu_lo),
// from the coefficient rows (times E^2).
__device__ __forceinline__ float cut_rate(const KParams& P, int m, const Phys& ph, float E, float s_c) {
    const float4* r = P.cut + (uint32_t)(m * P.N + ph.k) * 2u;
    float4 a = __ldg(r), b = __ldg(r + 1);
    float R = fmaf(a.y, ph.f, a.x), Hc = fmaf(a.w, ph.f, a.z), Hlo = fmaf(b.y, ph.f, b.x);
    float rate = R * (__fdividef(1.f, s_c) - 0.5f) - Hlo;
    if (Hc > 0.f) {
        float eta = (float)kFineStructure * rsqrtf(2.f * E / (float)kProtonMass);
        rate = fmaf(Hc, mott_prim(s_c, eta), rate);
    }
    return rate * __fdividef(1.f, E * E);
}

// ------------------------------------------------------------ jump samplers
// Identical-particle Coulomb law of hydrogen on [-cos(theta_b), cos(theta_c)]
// (CM cosine), inverted by Newton's method on its closed-form primitive
// G(mu) = 2 mu/(1-mu^2) - sin(eta ln((1+mu)/(1-mu)))/(2 eta), which is odd in
// mu: the root is sought in the forward variable s = 1 - |mu| and mirrored.
// Newton starts 13 % off at most and converges quadratically (1e-7 relative after four
// steps over 0.05-200 MeV); the fifth brings it to FP32 rounding.  The fast intrinsics
// keep the root within a few ulp: the arguments stay inside [-2 pi, 2 pi] for the
// fixed cut-off and the divisors far below 2^126.
__device__ void mott_sample(float U, float eta, float s_cut, float s_back, float& c, float& sn) {
    const float inv2eta = __fdividef(0.5f, eta);
    float g_hi = mott_prim(s_cut, eta), g_lo = -mott_prim(s_back, eta);
    float target = g_lo + U * (g_hi - g_lo);
    float sg = target >= 0.f ? 1.f : -1.f;
    float y = fabsf(target);
    float q = step_sqrt(1.f + y * y);
    float s = __fdividef(1.f + __fdividef(1.f, q + y), 1.f + q);  // root without the sine term
    float s_min = sg > 0.f ? s_cut : s_back;
#pragma unroll 1
    for (int it = 0; it < 5; ++it) {
        float mu = 1.f - s, rom2 = __fdividef(1.f, s * (2.f - s));
        float L = __logf(__fdividef(2.f - s, s));
        float sl, cl;
        __sincosf(eta * L, &sl, &cl);
        float G = 2.f * mu * rom2 - sl * inv2eta;
        float dG = (2.f * (1.f + mu * mu) * rom2 - cl) * rom2;
        s = fminf(fmaxf(s + __fdividef(G - y, dG), s_min), 1.f);
    }
    c = sg * (1.f - s);
    sn = step_sqrt(s * (2.f - s));
}

// The same law with the fixed cut-off, from tables: the primitive at the two ends of the
// range is interpolated in ln E, the root starts from the closed-form root s0 of the
// primitive without its sine term times the tabulated ratio rho(E, log2 s0) (bilinear,
// ~1e-4 relative), and one Newton step brings it to FP32 precision (the error squares).
__device__ __forceinline__ void mott_sample_tab(const KParams& P, float U, float eta, int k, float f, float& c,
                                                float& sn) {
    const float4 gt = __ldg(&P.mott_g[k]);
    const float g_hi = fmaf(gt.y, f, gt.x), g_lo = fmaf(gt.w, f, gt.z);
    const float target = g_lo + U * (g_hi - g_lo);
    const float sg = target >= 0.f ? 1.f : -1.f;
    const float y = fabsf(target);
    const float q = step_sqrt(1.f + y * y);
    const float s0 = __fdividef(1.f + __fdividef(1.f, q + y), 1.f + q);
    float jf = (__log2f(s0) - P.mott_lg2_lo) * P.mott_inv_dj;
    jf = fminf(fmaxf(jf, 0.f), (float)(kMottKnots - 1));
    const int j = min((int)jf, kMottKnots - 2);
    const float fj = jf - (float)j;
    const float2 r0 = __ldg(&P.mott_r[(uint32_t)(k * kMottKnots + j)]);
    const float2 r1 = __ldg(&P.mott_r[(uint32_t)((k + 1) * kMottKnots + j)]);
    const float ra = fmaf(r0.y - r0.x, fj, r0.x), rb = fmaf(r1.y - r1.x, fj, r1.x);
    const float s_min = sg > 0.f ? P.s_cut : P.s_back;
    float s = fminf(fmaxf(s0 * fmaf(rb - ra, f, ra), s_min), 1.f);
    {  // one Newton step on G(s) = y
        const float mu = 1.f - s, rom2 = __fdividef(1.f, s * (2.f - s));
        const float L = __logf(__fdividef(2.f - s, s));
        float sl, cl;
        __sincosf(eta * L, &sl, &cl);
        const float G = 2.f * mu * rom2 - sl * __fdividef(0.5f, eta);
        const float dG = (2.f * (1.f + mu * mu) * rom2 - cl) * rom2;
        s = fminf(fmaxf(s + __fdividef(G - y, dG), s_min), 1.f);
    }
    c = sg * (1.f - s);
    sn = step_sqrt(s * (2.f - s));
}

// Kalbach-Mann angular law a/(2 sinh a) (cosh(a mu) + r sinh(a mu)): the CDF
// is quadratic in T = exp(a mu); the stable root is taken on either sign of C.
__device__ float kalbach_mu(float U, float a, float r) {
    if (a < 1e-4f) return 2.f * U - 1.f;
    float ea = expf(a), eb = 1.f / ea;
    float sh = 0.5f * (ea - eb), ch = 0.5f * (ea + eb);
    float C = 2.f * sh * U + r * ch - sh;
    float q = sqrtf(C * C + (1.f - r) * (1.f + r));
    float T = C >= 0.f ? (C + q) / (1.f + r) : (1.f - r) / (q - C);
    return fminf(fmaxf(logf(T) / a, -1.f), 1.f);
}

// Kalbach (1988) slope parameter for proton in / proton out, separation
// energies neglected: e_a = E m2/(m_p+m2) (CM), e_b = (1-u) e_a.
__device__ float kalbach_a(float E, float u, float A) {
    float m2 = A * (float)kAtomicMassUnit;
    float ea = E * m2 / ((float)kProtonMass + m2);
    float X1 = fminf(ea, 130.f) * (1.f - u);
    float X3 = fminf(ea, 41.f) * (1.f - u);
    return 0.04f * X1 + 1.8e-6f * X1 * X1 * X1 + 6.7e-7f * (X3 * X3) * (X3 * X3);
}

// CM -> lab polar angle (Appendix A.1).  Elastic: v'_1C = p m2/(m_p^2 + E_tot m2)
// (the collinear Lorentz transform simplified); non-elastic: the printed
// collinear transform of the outgoing lab energy, used as a speed.
__device__ void cm_to_lab(float E, float Eout, bool elastic, float m2, float cc, float sc, float& cl,
                          float& sl) {
    const float mp = (float)kProtonMass;
    float p1 = step_sqrt(E * (E + 2.f * mp)), Et = E + mp;
    float ucm = p1 / (Et + m2);
    float gu = rsqrtf((1.f - ucm) * (1.f + ucm));
    float v;
    if (elastic) {
        v = __fdividef(p1 * m2, mp * mp + Et * m2);
    } else {
        float po = sqrtf(Eout * (Eout + 2.f * mp)), Eo = Eout + mp;
        v = fabsf(po - ucm * Eo) / (Eo - ucm * po);
    }
    float X = v * sc, Y = gu * (v * cc + ucm);
    float inv = rsqrtf(X * X + Y * Y);
    cl = Y * inv;
    sl = X * inv;
}

// Outcome of a large-angle event: the new direction, the refreshed clock, the factor
// (1 - u) on the post-loss energy (1 for elastic events) and the kind (1 elastic, 2
// non-elastic, 0 none).  Returned by value so that the caller's state stays in registers.
struct JumpOut {
    float ux, uy, uz, tau, e_fac;
    int kind;
    float uu;  // non-elastic loss fraction u (0 for elastic events)
    int el;    // element of the event
};

// A large-angle event of Eq. Npi at pre-step energy E (table interval k, fraction f):
// pick channel and element by rate, sample the CM angle, convert to the lab, rotate.
// sj = the step's total jump rate x Delta per unit density (the clock's rate), so the
// per-element rates need only be summed until the pick.
// CUT: the energy-dependent cut-off s_c = 1 - cos(theta_c) of this step (compiled
// separately so that the fixed-cut-off kernel carries none of it).
template <bool CUT>
__device__ __forceinline__ JumpOut do_jump(const KParams& P, int m, float E, int k, float f, uint4 J, float ux,
                                        float uy, float uz, float tau, uint64_t h, uint32_t n, float s_c,
                                        float sj, uint32_t segtag) {
    JumpOut o{ux, uy, uz, tau, 1.f, 0, 0.f, 0};
    const MatJump& mj = P.mats[m];
    const float* r0 = P.jrates + (uint32_t)(m * P.N + k) * (uint32_t)(2 * SDE_MAX_ELEMENTS);
    const float* r1 = r0 + 2 * SDE_MAX_ELEMENTS;
    const float rE2 = __fdividef(1.f, E * E);  // elastic rates are stored times E^2
    const float eta_h = (float)kFineStructure * rsqrtf(2.f * E / (float)kProtonMass);
    // The stored elastic rates are those of the fixed cut-off s_cut; with the variable
    // cut-off s_c they scale by the ratio of the angular factors (Rutherford: 1/s - 1/2,
    // hydrogen: G(s) - G(mu_lo)).
    float scale_R = rE2, scale_H = rE2;
    if (CUT) {
        scale_R *= (__fdividef(1.f, s_c) - 0.5f) / P.ruth_span;
        float glo = -mott_prim(P.s_back, eta_h);
        scale_H *= (mott_prim(s_c, eta_h) - glo) / (mott_prim(P.s_cut, eta_h) - glo);
    }
    int pick = -1;
    if (!CUT) {
        // Cumulative rows (per unit density, x Delta): the first channel whose cumulative rate
        // exceeds the target U sj.  Elastic rows are stored x E^2, so they are compared with
        // the target x E^2; the non-elastic rows with what remains of it.
        const float2* c = P.pick + (uint32_t)(m * P.N + k) * (uint32_t)(2 * SDE_MAX_ELEMENTS);
        const int ne = mj.n_el;
        const float t = u01(J.x) * sj;
        const float tE = t * (E * E);
        const float2 ce = c[ne - 1], cn = c[SDE_MAX_ELEMENTS + ne - 1];
        const float etot = fmaf(ce.y, f, ce.x), ntot = fmaf(cn.y, f, cn.x);
        if ((tE < etot && etot > 0.f) || !(ntot > 0.f)) {
            if (!(etot > 0.f)) return o;  // no channel open (cannot happen when the clock fired)
            int i = 0;
            while (i < ne - 1 && fmaf(c[i].y, f, c[i].x) <= tE) ++i;
            pick = i;
        } else {
            const float tn = fmaf(-etot, rE2, t);
            int i = 0;
            while (i < ne - 1 && fmaf(c[SDE_MAX_ELEMENTS + i].y, f, c[SDE_MAX_ELEMENTS + i].x) <= tn) ++i;
            pick = SDE_MAX_ELEMENTS + i;
        }
    } else {
        float target = u01(J.x) * (sj * P.inv_delta_cm), acc = 0.f;
        int last = -1;
        for (int ch = 0; ch < 2 && pick < 0; ++ch)
            for (int i = 0; i < mj.n_el; ++i) {
                int o = ch * SDE_MAX_ELEMENTS + i;
                float rate = fmaf(r1[o] - r0[o], f, r0[o]) * (ch == 0 ? (mj.Z[i] == 1 ? scale_H : scale_R) : 1.f);
                if (rate <= 0.f) continue;
                last = o;
                acc += rate;
                if (target < acc) {
                    pick = o;
                    break;
                }
            }
        if (pick < 0) pick = last;
        if (pick < 0) return o;  // no channel open (cannot happen when the clock fired)
    }
    int el = pick % SDE_MAX_ELEMENTS;
    bool elastic = pick < SDE_MAX_ELEMENTS;
    float m2 = mj.m2[el];
    float cc, sc, cl, sl;
    if (elastic) {
        if (mj.Z[el] == 1) {
            if (CUT)
                mott_sample(u01(J.y), eta_h, s_c, P.s_back, cc, sc);
            else
                mott_sample_tab(P, u01(J.y), eta_h, k, f, cc, sc);
        } else {
            float span = CUT ? __fdividef(1.f, s_c) - 0.5f : P.ruth_span;
            float s = __fdividef(1.f, 0.5f + u01(J.y) * span);
            cc = 1.f - s;
            sc = step_sqrt(s * (2.f - s));
        }
        cm_to_lab(E, E, true, m2, cc, sc, cl, sl);
    } else {
        uint4 J2 = philox(P, n, kTagJumpB | segtag, h);
        float uu = P.inel_lo + P.inel_span * u01(J.y);
        float mu = kalbach_mu(u01(J2.x), kalbach_a(E, uu, mj.A[el]), P.km_r);
        cc = mu;
        sc = sqrtf(fmaxf(0.f, (1.f - mu) * (1.f + mu)));
        cm_to_lab(E, E * (1.f - uu), false, m2, cc, sc, cl, sl);
        o.e_fac = 1.f - uu;
        o.uu = uu;
    }
    o.el = el;
    float sp, cp;
    __sincosf(kTwoPiF * u01(J.z), &sp, &cp);
    rotate(o.ux, o.uy, o.uz, cl, sl, cp, sp);
    o.tau = -__logf(u01(J.w));
    o.kind = elastic ? 1 : 2;
    return o;
}

// Continuous part of one Euler-Maruyama step of Eq. VSDE at Y_n = (E, ., u) in
// material m of density rho, with the step's Philox block x: on return E1 = energy
// after the continuous loss, u = direction after the Brownian increment, tau = the
// jump clock after the step, s_c = the step's elastic cut-off and ph = the table
// position of E.  The clock is exponential: tau ~ Exp(1) is spent at rate sigma per
// unit path; crossing zero within a step is the step's jump, which has probability
// 1 - exp(-Delta sigma) as in the paper.  Returns true when it crossed: the step then
// ends with a large-angle event (do_jump at the pre-step energy E).  Switched-off terms
// are multiplied by zero (no branches).
template <bool CUT>
__device__ __forceinline__ bool sde_step_cont(const KParams& P, const float4* tab, int m, float rho, uint4 x,
                                              float E, float& ux, float& uy, float& uz, float& tau,
                                              float& E1_out, float& s_c_out, Phys& ph_out, float& sj_out) {
    Phys ph = lookup(tab, P, m, E);
    float c = rho * ph.c;                   // varsigma_1 Delta
    float s = step_sqrt(rho) * ph.s * P.strag_on;  // varsigma_2 sqrt(Delta)
    float r = step_sqrt(-2.f * __logf(u01(x.x)));
    float zE = r * __cosf(kTwoPiF * u01(x.y));
    // The clamp keeps the energy non-increasing (Eq. VSDE); in FP32 (E - c) + c can
    // round one ulp above E, which would make the step's fixed-point deposit negative.
    float E1 = fminf(fmaxf(E - c + fminf(fmaxf(s * zE, -c), c), 0.f), E);
    // Lynch-Dahl: w = chi_c^2/(2 chi_alpha^2 (1-F)), sigma^2 = chi_c^2/(1+F^2) g(w),
    // g(w) = (1+w)/w ln(1+w) - 1; Brownian time t = sigma^2 Delta / z.
    float w = rho * ph.w;
    float g;
    if (w >= 1.f)
        g = __fdividef(1.f + w, w) * __logf(1.f + w) - 1.f;
    else if (w >= 0.01f)
        g = __fdividef(1.f + w, w) * log1pf(w) - 1.f;
    else
        g = w * (0.5f + w * (-1.f / 6.f + w * (1.f / 12.f)));
    const float t_raw = rho * ph.tg * g;  // sigma^2 Delta / z, whether or not scattering is on
    float t = t_raw * P.mcs_on;
    float th2 = -2.f * t * __logf(u01(x.z));
    float ct, st;
    cos_sin_from_sq(th2, ct, st);
    float sp, cp;
    __sincosf(kTwoPiF * u01(x.w), &sp, &cp);
    rotate(ux, uy, uz, ct, st, cp, sp);
    E1_out = E1;
    float sj = ph.sj, s_c = P.s_cut;
    if (CUT) {  // variable cut-off theta_c = k sigma(E): theta_c^2 = k^2 (z/Delta) t
        s_c = cut_s(P.cut_k2 * t_raw);
        sj = cut_rate(P, m, ph, E, s_c) + ph.sn;
    }
    s_c_out = s_c;
    sj_out = sj;
    ph_out = ph;
    tau -= rho * sj;
    return tau <= 0.f;
}

// The whole step (continuous part and, when the clock fires, the event at once).  On
// return E1 = energy after the continuous loss, E = energy after any non-elastic event,
// u = new direction; returns 0/1/2 (no jump, elastic, non-elastic).
template <bool CUT>
__device__ __forceinline__ int sde_step(const KParams& P, const float4* tab, int m, float rho, uint4 x,
                                        float& E, float& ux, float& uy, float& uz, float& tau, uint64_t h,
                                        uint32_t n, float& E1_out) {
    float E1, s_c, sj;
    Phys ph;
    int jump = 0;
    if (sde_step_cont<CUT>(P, tab, m, rho, x, E, ux, uy, uz, tau, E1, s_c, ph, sj)) {
        JumpOut o = do_jump<CUT>(P, m, E, ph.k, ph.f, philox(P, n, kTagJumpA, h), ux, uy, uz, tau, h, n, s_c, sj, 0u);
        ux = o.ux;
        uy = o.uy;
        uz = o.uz;
        tau = o.tau;
        jump = o.kind;
        E1_out = E1;
        E1 *= o.e_fac;
    } else {
        E1_out = E1;
    }
    E = E1;
    return jump;
}

// Sample Y_0 of history h from its spot (binary search of the history prefix).
#ifdef SDE_INIT_NOINLINE
#define SDE_INIT_ATTR __noinline__
#else
#define SDE_INIT_ATTR __forceinline__
#endif
__device__ SDE_INIT_ATTR void init_history(const KParams& P, uint64_t h, float& E, float& px, float& py,
                                             float& pz, float& ux, float& uy, float& uz, float& tau) {
    int lo = 0, hi = P.n_spots;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (P.prefix[mid] <= h)
            lo = mid;
        else
            hi = mid;
    }
    const SpotDev& s = P.spots[lo];
    uint4 A = philox(P, 0u, kTagSrcA, h);
    uint4 B = philox(P, 0u, kTagSrcB, h);
    float r = step_sqrt(-2.f * __logf(u01(A.x)));
    float sa, ca;
    __sincosf(kTwoPiF * u01(A.y), &sa, &ca);
    float g1 = r * ca, g2 = r * sa;
    float g3 = step_sqrt(-2.f * __logf(u01(A.z))) * __cosf(kTwoPiF * u01(A.w));
    E = fminf(fmaxf(s.E + s.sE * g3, P.e_min), P.e_max);
    px = fmaf(g1, s.e1x, fmaf(g2, s.e2x, s.px));  // voxel units (the basis carries sigma / h)
    py = fmaf(g1, s.e1y, fmaf(g2, s.e2y, s.py));
    pz = fmaf(g1, s.e1z, fmaf(g2, s.e2z, s.pz));
    ux = s.ux;
    uy = s.uy;
    uz = s.uz;
    if (s.sang > 0.f) {
        float th2 = -2.f * __logf(u01(B.x)) * s.sang * s.sang;
        float ct, st, sp, cp;
        cos_sin_from_sq(th2, ct, st);
        __sincosf(kTwoPiF * u01(B.y), &sp, &cp);
        rotate(ux, uy, uz, ct, st, cp, sp);
    }
    tau = -__logf(u01(B.z));
}

// Branching model: the secondary proton of a primary's non-elastic event (its j-th), in
// the order of the oracle: energy kappa u E1 (E1 = the primary's post-loss energy), a
// Kalbach-Mann CM angle at slope a(E_n, 1 - kappa u) converted to the lab with outgoing
// energy kappa u E_n, about the incoming (diffused) direction, uniform azimuth, a fresh
// clock; draws y, z, w of the event's second Philox block.  Starts at the primary's
// position R_{n+1}.  Pushed to the queue; returns its energy in tally units, or 0 when the
// queue is full (the caller then counts that energy as removed and the flag is raised).
__device__ __noinline__ unsigned long long spawn_secondary(const KParams& P, int m, int el, float En, float E1,
                                                           float uu, float ux, float uy, float uz, float px,
                                                           float py, float pz, uint64_t h, uint32_t n,
                                                           uint32_t j) {
    const MatJump& mj = P.mats[m];
    const float ks = P.sec_frac * uu;
    const float Es = ks * E1;
    const uint4 J2 = philox(P, n, kTagJumpB, h);
    const float mu = kalbach_mu(u01(J2.y), kalbach_a(En, 1.f - ks, mj.A[el]), P.km_r);
    float cl, sl;
    cm_to_lab(En, En * ks, false, mj.m2[el], mu, sqrtf(fmaxf(0.f, (1.f - mu) * (1.f + mu))), cl, sl);
    float sp, cp;
    __sincosf(kTwoPiF * u01(J2.z), &sp, &cp);
    rotate(ux, uy, uz, cl, sl, cp, sp);
    const unsigned long long slot = atomicAdd(P.sec_ctl, 1ull);
    if (slot >= P.sec_cap) {
        atomicOr(P.err, kErrSecQueue);
        return 0ull;
    }
    SecRec r;
    r.h = h;
    r.seg = j;
    r.E = Es;
    r.px = px;
    r.py = py;
    r.pz = pz;
    r.ux = ux;
    r.uy = uy;
    r.uz = uz;
    r.tau = -__logf(u01(J2.w));
    r.pad = 0u;
    P.sec_q[slot] = r;
    return qfix(P, Es);
}

// Voxel containing a point given in voxel units (floor convention; -1 outside).
__device__ __forceinline__ int voxel_index(const KParams& P, float gx, float gy, float gz) {
    int ix = __float2int_rd(gx);
    int iy = __float2int_rd(gy);
    int iz = __float2int_rd(gz);
    if ((unsigned)ix >= (unsigned)P.nx || (unsigned)iy >= (unsigned)P.ny || (unsigned)iz >= (unsigned)P.nz)
        return -1;
    return ix + P.nx * (iy + P.ny * iz);
}

// Packed voxel word: density (FP32, low 4 mantissa bits rounded away) with the
// material id in those 4 bits.
__device__ __forceinline__ int vox_mat(uint32_t w) { return (int)(w & 15u); }
__device__ __forceinline__ float vox_rho(uint32_t w) { return __uint_as_float(w & ~15u); }

// Split dq along the chord (ax,ay,az) + t (dx,dy,dz), t in [0,1] (voxel units), over
// the voxels it crosses, in proportion to the length inside each (Amanatides-Woo
// traversal).  Pieces are cumulative roundings of t dq, so they sum to dq.
// Returns the part that falls outside the grid.
__device__ unsigned long long deposit_chord(const KParams& P, float ax, float ay, float az, float dx,
                                            float dy, float dz, unsigned long long dq) {
    float g[3] = {ax, ay, az};
    float v[3] = {dx, dy, dz};
    int n[3] = {P.nx, P.ny, P.nz};
    int i[3], st[3];
    float tmax[3], tdel[3];
    for (int a = 0; a < 3; ++a) {
        i[a] = __float2int_rd(g[a]);
        if (v[a] > 0.f) {
            st[a] = 1;
            tmax[a] = ((float)(i[a] + 1) - g[a]) / v[a];
            tdel[a] = 1.f / v[a];
        } else if (v[a] < 0.f) {
            st[a] = -1;
            tmax[a] = ((float)i[a] - g[a]) / v[a];
            tdel[a] = -1.f / v[a];
        } else {
            st[a] = 0;
            tmax[a] = INFINITY;
            tdel[a] = INFINITY;
        }
    }
    float fq = (float)dq;
    unsigned long long done = 0, escaped = 0;
    for (int it = 0; it < 32 && done < dq; ++it) {
        float tn = fminf(fminf(tmax[0], tmax[1]), tmax[2]);
        bool last = tn >= 1.f || it == 31;
        unsigned long long upto = last ? dq : __float2ull_rn(tn * fq);
        upto = upto < done ? done : (upto > dq ? dq : upto);
        unsigned long long part = upto - done;
        done = upto;
        if (part) {
            bool in = (unsigned)i[0] < (unsigned)n[0] && (unsigned)i[1] < (unsigned)n[1] &&
                      (unsigned)i[2] < (unsigned)n[2];
            if (in)
                atomicAdd(&P.edep[i[0] + P.nx * (i[1] + P.ny * i[2])], part);
            else
                escaped += part;
        }
        if (last) break;
        int ax_ = (tmax[0] <= tmax[1] && tmax[0] <= tmax[2]) ? 0 : (tmax[1] <= tmax[2] ? 1 : 2);
        i[ax_] += st[ax_];
        tmax[ax_] += tdel[ax_];
    }
    return escaped;
}

// Four resident blocks of 256 threads per SM: 64 registers per thread, enough for the
// step body without spills.  Measured against 48 registers (five blocks, spilled loop
// state), 40 (six blocks) and 56, 72 and 76 registers: the unspilled 64 was fastest by
// 2-3 %, with bit-identical tallies.
#ifndef SDE_MIN_BLOCKS
#define SDE_MIN_BLOCKS 4
#endif


// Rare events (start, escape, non-elastic removal, jumps) go to per-block
// shared-memory counters; the per-step deposit needs no counter at all: the
// deposited total is the sum of the tally, reduced when the balance is read.
#define SDE_BLOCK_ADD(idx, v) atomicAdd(&s_cnt[idx], (unsigned long long)(v))

// BR: 0 plain transport; 1 primaries that queue the secondaries of the branching model;
// 2 the queued secondaries (work items are queue records, not history ids).
template <int TALLY, bool SMEM, bool AGG, bool CUT, int BR>
__global__ void __launch_bounds__(256, SDE_MIN_BLOCKS) k_transport(const __grid_constant__ KParams P) {
    extern __shared__ float4 s_tab[];
    __shared__ unsigned long long s_cnt[kCntWords];
    // The warp's current batch of history ids [next, end) is warp-uniform: it lives in
    // shared memory, not in four registers of every lane.
    __shared__ unsigned long long s_batch[2 * kMaxWarpsPerBlock];
    if (threadIdx.x < kCntWords) s_cnt[threadIdx.x] = 0ull;
    if (threadIdx.x < 2 * kMaxWarpsPerBlock) s_batch[threadIdx.x] = 0ull;
    const float4* tab = P.table;
    if (SMEM) {
        int rows = P.n_mats * P.N * kRowFloat4;
        for (int i = threadIdx.x; i < rows; i += blockDim.x) s_tab[i] = P.table[i];
        tab = s_tab;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    unsigned long long total = P.prefix[P.n_spots] < P.h_end ? P.prefix[P.n_spots] : P.h_end;
    if (BR == 2) total = P.sec_ctl[0] < P.sec_cap ? P.sec_ctl[0] : P.sec_cap;
    unsigned long long* const cursor = BR == 2 ? &P.sec_ctl[1] : &P.counters[kCntCursor];
    bool alive = false;
    // position (voxel units) and direction; x and y as pairs for packed FP32x2 arithmetic
    float2 pxy = make_float2(0.f, 0.f), uxy = make_float2(0.f, 0.f);
    float E = 0.f, pz = 0.f, uz = 1.f, tau = 1.f;
    unsigned long long h = 0;
    uint32_t n = 0;
    uint32_t segtag = 0;  // BR 2: the track's segment index << 8 (Philox tag bits)
    uint32_t nsec = 0;    // BR 1: non-elastic events of the primary so far
    // Pending large-angle event of step n - 1: the material of that step (-1: none),
    // its pre-step energy, its cut-off and its total jump rate.
    int jm = -1;
    float jE = 0.f, jsc = 0.f, jsj = 0.f;
    // Software pipeline: the voxel word of R_n and the Philox block of step n are
    // fetched/computed during step n-1, so their latency overlaps the step's work.
    uint32_t vox = 0;
    int vcur = -1;
    uint4 x = make_uint4(0u, 0u, 0u, 0u);
    unsigned long long* const s_next = &s_batch[2 * (threadIdx.x >> 5)];
    unsigned long long* const s_end = s_next + 1;
    bool drained = false;

    for (;;) {
        unsigned dead = __ballot_sync(0xffffffffu, !alive);
        // refill when the whole warp is idle, or at least refill_min lanes are; once
        // started, until every lane is busy or the queue is drained
        if (dead == 0xffffffffu || (dead && __popc(dead) >= P.refill_min)) {
            while (dead && !drained) {
                unsigned long long b_next = *s_next, b_end = *s_end;
                if (b_next >= b_end) {
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(cursor, (unsigned long long)P.batch);
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (base >= total) {
                        drained = true;
                        break;
                    }
                    b_next = base;
                    b_end = min(base + (unsigned long long)P.batch, total);
                }
                int nd = __popc(dead);
                unsigned long long avail = b_end - b_next;
                int take = (unsigned long long)nd < avail ? nd : (int)avail;
                int rank = __popc(dead & ((1u << lane) - 1u));
                if (((dead >> lane) & 1u) && rank < take) {
                    n = 0;
                    alive = true;
                    if (BR == 2) {
                        const SecRec& r = P.sec_q[b_next + (unsigned long long)rank];
                        h = r.h;
                        segtag = r.seg << 8;
                        E = r.E;
                        pxy = make_float2(r.px, r.py);
                        pz = r.pz;
                        uxy = make_float2(r.ux, r.uy);
                        uz = r.uz;
                        tau = r.tau;
                    } else {
                        h = b_next + (unsigned long long)rank;
                        init_history(P, h, E, pxy.x, pxy.y, pz, uxy.x, uxy.y, uz, tau);
                        SDE_BLOCK_ADD(kCntIncident, qfix(P, E));
                        SDE_BLOCK_ADD(kCntHistories, 1);
                        nsec = 0;
                    }
                    vcur = voxel_index(P, pxy.x, pxy.y, pz);
                    vox = vcur >= 0 ? __ldg(&P.vox[vcur]) : 0u;
                    x = philox(P, 0u, kTagStep | segtag, h);
                    if (BR == 2 && E < P.e_min) {  // emitted below the absorption energy
                        unsigned long long qr = qfix(P, E);
                        if (qr) {
                            if (vcur >= 0)
                                atomicAdd(&P.edep[vcur], qr);
                            else
                                SDE_BLOCK_ADD(kCntEscaped, qr);
                        }
                        alive = false;
                    }
                }
                b_next += (unsigned long long)take;
                __syncwarp();
                if (lane == 0) {
                    *s_next = b_next;
                    *s_end = b_end;
                }
                __syncwarp();
                dead = __ballot_sync(0xffffffffu, !alive);
            }
        }
        if (dead == 0xffffffffu) break;  // queue drained and every lane idle
        // A large-angle event whose clock fired in the previous step is sampled here,
        // outside the step body, before the history's next step; each history keeps its
        // own order of operations and random numbers.
        if (jm >= 0) {
            int k;
            float f;
            grid_pos(P, jE, k, f);  // the table position the step's lookup used
            const uint32_t nj = n - 1u;
            JumpOut o = do_jump<CUT>(P, jm, jE, k, f, philox(P, nj, kTagJumpA | segtag, h), uxy.x, uxy.y, uz,
                                     tau, h, nj, jsc, jsj, segtag);
            unsigned long long q_sec = 0;
            if (BR == 1 && o.kind == 2)  // the secondary leaves the incoming direction at R_{n+1}
                q_sec = spawn_secondary(P, jm, o.el, jE, E, o.uu, uxy.x, uxy.y, uz, pxy.x, pxy.y, pz, h, nj,
                                        ++nsec);
            uxy = make_float2(o.ux, o.uy);
            uz = o.uz;
            tau = o.tau;
            jm = -1;
            if (o.kind == 2) {
                const float Ej = E * o.e_fac;  // E is still the step's post-loss energy E1
                // the deficit leaves the transport except what a secondary carries on (the
                // three terms are roundings; their sum over a launch is exact modulo 2^64)
                SDE_BLOCK_ADD(kCntRemoved, qfix(P, E) - qfix(P, Ej) - q_sec);
                SDE_BLOCK_ADD(kCntJumpInel, 1);
                E = Ej;
            } else if (o.kind == 1) {
                SDE_BLOCK_ADD(kCntJumpEl, 1);
            }
            if (E < P.e_min) {  // absorbed, as at the end of a step
                unsigned long long qr = qfix(P, E);
                if (qr) {
                    if (vcur >= 0)
                        atomicAdd(&P.edep[vcur], qr);
                    else
                        SDE_BLOCK_ADD(kCntEscaped, qr);
                }
                SDE_BLOCK_ADD(kCntSteps, n);
                alive = false;
            }
        }
        if (!alive) continue;

        if (n >= (uint32_t)P.max_steps || vcur < 0) {  // step cap, or R_n outside the domain D
            if (n >= (uint32_t)P.max_steps) atomicOr(P.err, kErrStepCap);
            SDE_BLOCK_ADD(kCntEscaped, qfix(P, E));
            SDE_BLOCK_ADD(kCntSteps, n);
            alive = false;
            continue;
        }
        const int m = vox_mat(vox);
        const float rho = vox_rho(vox);
        // Position line of Eq. VSDE along the pre-step direction; the next voxel word
        // is requested now and consumed by the next step.
        const float2 oxy = pxy, ouxy = uxy;
        const float oz = pz, ouz = uz;
        pxy = __ffma2_rn(ouxy, P.sv_xy, pxy);
        pz = fmaf(ouz, P.sv_z, pz);
        const int vnext = voxel_index(P, pxy.x, pxy.y, pz);
        const uint32_t vox_next = vnext >= 0 ? __ldg(&P.vox[vnext]) : 0u;
        const uint4 xcur = x;
        x = philox(P, n + 1u, kTagStep | segtag, h);
        const unsigned long long q0 = qfix(P, E);
        float E1, s_c, sj;
        Phys ph;
        const bool fired = sde_step_cont<CUT>(P, tab, m, rho, xcur, E, uxy.x, uxy.y, uz, tau, E1, s_c, ph, sj);
        if (fired) {  // the event waits; the step's deposit does not depend on it
            jm = m;
            jE = E;
            jsc = s_c;
            jsj = sj;
        }
        E = E1;
        unsigned long long q1 = qfix(P, E1);
        unsigned long long dq = q0 - q1;
        if (TALLY == 0) {
            // deposit at the step midpoint (Sec. 2.2.2)
            const float2 mxy = __ffma2_rn(ouxy, P.hv_xy, oxy);
            int mv = voxel_index(P, mxy.x, mxy.y, fmaf(ouz, P.hv_z, oz));
            if (mv < 0) {
                if (dq) SDE_BLOCK_ADD(kCntEscaped, dq);
            } else if (AGG) {
                // Lanes depositing into the same voxel add their parts first and one
                // lane commits the sum.  dq < 2^40 (E <= 1000 MeV in units of at least
                // 2^-30 MeV), so the sums of the 24-bit low parts and of the high parts
                // of up to 32 lanes each fit 32 bits and the 64-bit sum is exact.
                unsigned grp = __match_any_sync(__activemask(), mv);
                unsigned lo = __reduce_add_sync(grp, (unsigned)(dq & 0xFFFFFFull));
                unsigned hi = __reduce_add_sync(grp, (unsigned)(dq >> 24));
                unsigned long long sum = ((unsigned long long)hi << 24) + lo;
                if (lane == __ffs(grp) - 1 && sum) atomicAdd(&P.edep[mv], sum);
            } else if (dq) {
                atomicAdd(&P.edep[mv], dq);
            }
        } else if (dq) {
            const float2 dxy = __fmul2_rn(ouxy, P.sv_xy);
            unsigned long long esc = deposit_chord(P, oxy.x, oxy.y, oz, dxy.x, dxy.y, ouz * P.sv_z, dq);
            if (esc) SDE_BLOCK_ADD(kCntEscaped, esc);
        }
        n += 1;
        vcur = vnext;
        vox = vox_next;
        if (!fired && E < P.e_min) {  // absorbed; the rest is deposited where the proton is
            unsigned long long qr = qfix(P, E);
            if (qr) {
                if (vcur >= 0)
                    atomicAdd(&P.edep[vcur], qr);
                else
                    SDE_BLOCK_ADD(kCntEscaped, qr);
            }
            SDE_BLOCK_ADD(kCntSteps, n);  // the history's steps, counted once at its end
            alive = false;
        }
    }

    __syncthreads();
    if (threadIdx.x < kCntWords && threadIdx.x != kCntCursor && threadIdx.x != kCntDeposited &&
        s_cnt[threadIdx.x])
        atomicAdd(&P.counters[threadIdx.x], s_cnt[threadIdx.x]);
}
#undef SDE_BLOCK_ADD

// Sum of the tally (the deposited energy of the balance), added to *out.
__global__ void k_sum_u64(const unsigned long long* __restrict__ v, size_t n, unsigned long long* out) {
    unsigned long long acc = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        acc += v[i];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

// Spot records -> device form and the inclusive prefix of history counts;
// sets the work-queue cursor to the first history id of the run.  One block.
__global__ void __launch_bounds__(1024) k_prep_spots(const sde_spot* raw, int n, SpotDev* out,
                                                     unsigned long long* prefix,
                                                     unsigned long long* counters, unsigned int* err,
                                                     double ox, double oy, double oz, double ihx, double ihy,
                                                     double ihz, double e_min, double e_lim,
                                                     unsigned long long h_begin) {
    __shared__ unsigned long long scan[1024];
    unsigned long long carry = 0;
    for (int base = 0; base < n; base += blockDim.x) {
        int i = base + threadIdx.x;
        unsigned long long nh = 0;
        if (i < n) {
            sde_spot s = raw[i];
            double un = s.ux * s.ux + s.uy * s.uy + s.uz * s.uz;
            bool ok = s.E_MeV > e_min && s.E_MeV + 5.0 * s.sigma_E_MeV <= e_lim && s.sigma_E_MeV >= 0.0 &&
                      s.sigma_xy_mm >= 0.0 && s.sigma_xy_mm < 1e4 && s.sigma_angle_rad >= 0.0 &&
                      s.sigma_angle_rad < 1.0 && un > 0.0 && isfinite(un) && isfinite(s.x_mm) &&
                      isfinite(s.y_mm) && isfinite(s.z_mm);
            SpotDev d = {};
            if (ok) {
                nh = s.n_hist;
                double inv = rsqrt(un);
                double x = s.ux * inv, y = s.uy * inv, z = s.uz * inv;
                double sg = copysign(1.0, z);
                double a = -1.0 / (sg + z), b = x * y * a;
                d.E = (float)s.E_MeV;
                d.sE = (float)s.sigma_E_MeV;
                d.sxy = (float)s.sigma_xy_mm;
                d.sang = (float)s.sigma_angle_rad;
                const double sx = s.sigma_xy_mm * ihx, sy = s.sigma_xy_mm * ihy, sz = s.sigma_xy_mm * ihz;
                d.px = (float)((s.x_mm - ox) * ihx);
                d.py = (float)((s.y_mm - oy) * ihy);
                d.pz = (float)((s.z_mm - oz) * ihz);
                d.ux = (float)x;
                d.uy = (float)y;
                d.uz = (float)z;
                d.e1x = (float)((1.0 + sg * x * x * a) * sx);
                d.e1y = (float)(sg * b * sy);
                d.e1z = (float)(-sg * x * sz);
                d.e2x = (float)(b * sx);
                d.e2y = (float)((sg + y * y * a) * sy);
                d.e2z = (float)(-y * sz);
            } else {
                atomicOr(err, kErrBadSpot);
            }
            out[i] = d;
        }
        scan[threadIdx.x] = nh;
        __syncthreads();
        for (int off = 1; off < (int)blockDim.x; off <<= 1) {
            unsigned long long add = threadIdx.x >= (unsigned)off ? scan[threadIdx.x - off] : 0ull;
            __syncthreads();
            scan[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < n) prefix[i + 1] = carry + scan[threadIdx.x];
        carry += scan[blockDim.x - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        prefix[0] = 0;
        counters[kCntCursor] = h_begin;
    }
}

__global__ void k_probe(const __grid_constant__ KParams P, int m, float rho, float E0, uint64_t h0, int n, float* Eo, float* co,
                        int* jo, float* uxo, float* uyo) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t h = h0 + (uint64_t)i;
    uint4 B = philox(P, 0u, kTagSrcB, h);
    float tau = -__logf(u01(B.z));
    float E = E0, ux = 0.f, uy = 0.f, uz = 1.f, E1;
    int j = P.cut_k2 > 0.f
                ? sde_step<true>(P, P.table, m, rho, philox(P, 0u, kTagStep, h), E, ux, uy, uz, tau, h, 0u, E1)
                : sde_step<false>(P, P.table, m, rho, philox(P, 0u, kTagStep, h), E, ux, uy, uz, tau, h, 0u, E1);
    Eo[i] = E;
    co[i] = uz;
    jo[i] = j;
    uxo[i] = ux;
    uyo[i] = uy;
}

// Dose to medium (Sec. 2.2.2): tally units -> J over voxel mass (kg).  The FP64 unit of
// this GPU is narrow and a double division is a long sequence on it, so 1/mass is the
// FP32 reciprocal refined by one Newton step in FP64 (relative error ~1e-14).
template <typename T>
__global__ void k_convert(const unsigned long long* edep, const float* rho, size_t nv, double unit_J,
                          double vol_kg_per_rho, T* dose) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nv; v += (size_t)gridDim.x * blockDim.x) {
        const float r = rho[v];
        double out = 0.0;
        if (r > 0.f) {
            const double mass = (double)r * vol_kg_per_rho;
            double y = (double)__frcp_rn(__double2float_rn(mass));
            y = fma(y, fma(-mass, y, 1.0), y);
            out = (double)edep[v] * unit_J * y;
        }
        dose[v] = (T)out;
    }
}

// ---------------------------------------------------------------- launchers
template <int TALLY, bool SMEM, bool AGG, bool CUT, int BR>
static cudaError_t allow_smem(size_t smem) {
    if (!SMEM) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_transport<TALLY, SMEM, AGG, CUT, BR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
#ifdef SDE_SMEM_CARVEOUT
    e = cudaFuncSetAttribute(k_transport<TALLY, SMEM, AGG, CUT, BR>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             SDE_SMEM_CARVEOUT);
#endif
    return e;
}

template <int TALLY, bool SMEM, bool AGG, bool CUT, int BR = 0>
static cudaError_t launch_t(const KParams& P, int grid, int block, size_t smem, cudaStream_t st) {
    cudaError_t e = allow_smem<TALLY, SMEM, AGG, CUT, BR>(smem);
    if (e != cudaSuccess) return e;
    k_transport<TALLY, SMEM, AGG, CUT, BR><<<grid, block, SMEM ? smem : 0, st>>>(P);
    return cudaGetLastError();
}

template <int TALLY, bool SMEM, bool AGG, bool CUT, int BR = 0>
static int blocks_per_sm_t(int block, size_t smem) {
    if (allow_smem<TALLY, SMEM, AGG, CUT, BR>(smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_transport<TALLY, SMEM, AGG, CUT, BR>, block,
                                                      SMEM ? smem : 0) != cudaSuccess)
        return 0;
    return nb;
}

// Branching-model kernels: tables through L1 and per-lane atomics, either tally mode and
// either cut-off; BR 1 (primaries) or 2 (queued secondaries).
template <int BR>
static cudaError_t launch_branch(const KParams& P, int grid, int block, cudaStream_t st) {
    if (P.cut_k2 > 0.f)
        return P.tally_mode == 1 ? launch_t<1, false, false, true, BR>(P, grid, block, 0, st)
                                 : launch_t<0, false, false, true, BR>(P, grid, block, 0, st);
    return P.tally_mode == 1 ? launch_t<1, false, false, false, BR>(P, grid, block, 0, st)
                             : launch_t<0, false, false, false, BR>(P, grid, block, 0, st);
}

// Variant selection: tally mode (midpoint, chord), table placement, and warp
// aggregation of the tally; the energy-dependent cut-off has its own kernels (midpoint
// or chord tally, tables through L1, per-lane atomics) so that the fixed-cut-off ones
// carry none of its arithmetic; so has the branching model.
cudaError_t launch_transport(const KParams& P, int grid, int block, size_t smem_table, bool use_smem,
                             cudaStream_t st) {
    if (P.branch == 1) return launch_branch<1>(P, grid, block, st);
    if (P.branch == 2) return launch_branch<2>(P, grid, block, st);
    if (P.cut_k2 > 0.f)
        return P.tally_mode == 1 ? launch_t<1, false, false, true>(P, grid, block, 0, st)
                                 : launch_t<0, false, false, true>(P, grid, block, 0, st);
    if (P.tally_mode == 1)
        return use_smem ? launch_t<1, true, false, false>(P, grid, block, smem_table, st)
                        : launch_t<1, false, false, false>(P, grid, block, 0, st);
    if (P.aggregate)
        return use_smem ? launch_t<0, true, true, false>(P, grid, block, smem_table, st)
                        : launch_t<0, false, true, false>(P, grid, block, 0, st);
    return use_smem ? launch_t<0, true, false, false>(P, grid, block, smem_table, st)
                    : launch_t<0, false, false, false>(P, grid, block, 0, st);
}

int transport_max_blocks_per_sm(int block, size_t smem, bool use_smem, int tally_mode, bool aggregate, bool cut,
                                int branch) {
    if (branch) {
        // the primary and secondary kernels of one configuration run with one grid
        int a, b;
        if (cut) {
            a = tally_mode == 1 ? blocks_per_sm_t<1, false, false, true, 1>(block, 0)
                                : blocks_per_sm_t<0, false, false, true, 1>(block, 0);
            b = tally_mode == 1 ? blocks_per_sm_t<1, false, false, true, 2>(block, 0)
                                : blocks_per_sm_t<0, false, false, true, 2>(block, 0);
        } else {
            a = tally_mode == 1 ? blocks_per_sm_t<1, false, false, false, 1>(block, 0)
                                : blocks_per_sm_t<0, false, false, false, 1>(block, 0);
            b = tally_mode == 1 ? blocks_per_sm_t<1, false, false, false, 2>(block, 0)
                                : blocks_per_sm_t<0, false, false, false, 2>(block, 0);
        }
        return a < b ? a : b;
    }
    if (cut)
        return tally_mode == 1 ? blocks_per_sm_t<1, false, false, true>(block, 0)
                               : blocks_per_sm_t<0, false, false, true>(block, 0);
    if (tally_mode == 1)
        return use_smem ? blocks_per_sm_t<1, true, false, false>(block, smem)
                        : blocks_per_sm_t<1, false, false, false>(block, 0);
    if (aggregate)
        return use_smem ? blocks_per_sm_t<0, true, true, false>(block, smem)
                        : blocks_per_sm_t<0, false, true, false>(block, 0);
    return use_smem ? blocks_per_sm_t<0, true, false, false>(block, smem)
                    : blocks_per_sm_t<0, false, false, false>(block, 0);
}

// Start of one chunk of the branching model: the work-queue cursor at the chunk's first
// history id and an empty secondary queue.
__global__ void k_branch_chunk(unsigned long long* counters, unsigned long long* sec_ctl,
                               unsigned long long h_begin) {
    counters[kCntCursor] = h_begin;
    sec_ctl[0] = 0ull;
    sec_ctl[1] = 0ull;
}

cudaError_t launch_branch_chunk(unsigned long long* counters, unsigned long long* sec_ctl,
                                unsigned long long h_begin, cudaStream_t st) {
    k_branch_chunk<<<1, 1, 0, st>>>(counters, sec_ctl, h_begin);
    return cudaGetLastError();
}

cudaError_t launch_prep(const sde_spot* raw, int n, SpotDev* out, unsigned long long* prefix,
                        unsigned long long* counters, unsigned int* err, const double o[3], const double h[3],
                        double e_min, double e_lim, cudaStream_t st, unsigned long long h_begin) {
    k_prep_spots<<<1, 1024, 0, st>>>(raw, n, out, prefix, counters, err, o[0], o[1], o[2], 1.0 / h[0], 1.0 / h[1],
                                     1.0 / h[2], e_min, e_lim, h_begin);
    return cudaGetLastError();
}

cudaError_t launch_probe(const KParams& P, int m, float rho, float E0, uint64_t h0, int n, float* Eo,
                         float* co, int* jo, float* uxo, float* uyo, cudaStream_t st) {
    int threads = 256, blocks = (n + threads - 1) / threads;
    k_probe<<<blocks, threads, 0, st>>>(P, m, rho, E0, h0, n, Eo, co, jo, uxo, uyo);
    return cudaGetLastError();
}

cudaError_t launch_sum_u64(const unsigned long long* v, size_t n, unsigned long long* out, int num_sms,
                           cudaStream_t st) {
    k_sum_u64<<<num_sms * 4, 256, 0, st>>>(v, n, out);
    return cudaGetLastError();
}

cudaError_t launch_convert(const unsigned long long* edep, const float* rho, size_t nv, double unit_J,
                           double vol_kg_per_rho, double* dose, int num_sms, cudaStream_t st) {
    int blocks = num_sms * 4;
    k_convert<double><<<blocks, 256, 0, st>>>(edep, rho, nv, unit_J, vol_kg_per_rho, dose);
    return cudaGetLastError();
}

cudaError_t launch_convert_f32(const unsigned long long* edep, const float* rho, size_t nv, double unit_J,
                               double vol_kg_per_rho, float* dose, int num_sms, cudaStream_t st) {
    int blocks = num_sms * 4;
    k_convert<float><<<blocks, 256, 0, st>>>(edep, rho, nv, unit_J, vol_kg_per_rho, dose);
    return cudaGetLastError();
}

}  // namespace sde
