// Step body with two cells per thread and packed FP32 arithmetic (the f32x2
// add, multiply and fused multiply-add of sm_100 and later: one instruction
// computes the same operation for both cells, each element rounded as its
// scalar counterpart would be).  Used for FP32 arithmetic (FP32, FP16 and
// BF16 storage); FP64 keeps one cell per thread.
//
// A thread owns the adjacent cells x0 = 2t and x0 + 1 of one row, so the
// populations of both come from one aligned 8-byte (FP32) or 4-byte (16-bit)
// word wherever the direction does not move along x; an x-moving direction
// pulls its two cells from x0 - 1, x0 (c_x = +1) or x0 + 1, x0 + 2
// (c_x = -1) with two scalar loads.  Both cells share the row's table, its
// references and its index arithmetic.  The second cell of the last pair
// of an odd row lies in the row padding: it is computed from in-bounds
// values and stored there (nothing reads it), never summed.
//
// The arithmetic is that of step_body (moments, interface friction from
// lagged velocities, trapezoidal electron-phonon friction and sinks, Guo
// velocity, BGK + Guo collision with the FP32 moment fix-up), with the
// collision evaluated per pair of opposite directions: for c_ibar = -c_i the
// equilibrium and forcing terms split into parts even and odd in c,
//   teq = e0 + 4.5 rho (c.u)^2  +-  3 rho (c.u),
//   tF  = -3 u.F + 9 (c.u)(c.F) +-  3 (c.F),
// computed once per pair.

#pragma once

namespace klb {

__device__ __forceinline__ float2 b2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b, rounded once (b * -1 is exact).
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, b2(-1.f), a); }

// Pair access to the storage types.
template <typename S> struct Pair;
template <> struct Pair<float> {
    __device__ static float2 load2(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
    __device__ static float load1(const float *p) { return __ldg(p); }
    __device__ static void store2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
};
template <> struct Pair<__half> {
    __device__ static float2 load2(const __half *p)
    {
        return __half22float2(__ldg(reinterpret_cast<const __half2 *>(p)));
    }
    __device__ static float load1(const __half *p) { return Storage<__half>::load(p); }
    __device__ static void store2(__half *p, float2 v) { *reinterpret_cast<unsigned *>(p) = f32x2_to_f16x2_sat(v); }
};
template <> struct Pair<__nv_bfloat16> {
    __device__ static float2 load2(const __nv_bfloat16 *p)
    {
        return __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162 *>(p)));
    }
    __device__ static float load1(const __nv_bfloat16 *p) { return Storage<__nv_bfloat16>::load(p); }
    __device__ static void store2(__nv_bfloat16 *p, float2 v)
    {
        *reinterpret_cast<unsigned *>(p) = f32x2_to_bf16x2_sat(v);
    }
};

struct Cell2 {
    float2 drho;
    float2 u[3];
    float2 F[3];
};

// Source columns of the two cells for the three x shifts.
struct Cols {
    int x0, pm_a, pp_a, pp_b;
};

template <int Q>
__host__ __device__ constexpr int opp(int i)
{
    return dir_index<Q>(-cx<Q>(i), -cy<Q>(i), -cz<Q>(i));
}

// c_i . v for a pair of cells.
template <int Q>
__device__ __forceinline__ float2 cdot2(int i, const float2 v[3])
{
    const int c[3] = {cx<Q>(i), cy<Q>(i), cz<Q>(i)};
    float2 r = b2(0.f);
    bool any = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (c[a] == 0) continue;
        if (!any)
            r = c[a] > 0 ? v[a] : make_float2(-v[a].x, -v[a].y);
        else
            r = c[a] > 0 ? add2(r, v[a]) : sub2(r, v[a]);
        any = true;
    }
    return r;
}

// Mass and momentum of a population set, summed through the pairs of
// opposite directions (s = g_i + g_ibar, d = g_i - g_ibar) in shallow trees,
// so that the sums are short dependency chains.
template <int Q>
__device__ __forceinline__ void moments2(const float2 g[Q], float2 &m, float2 j[3])
{
    if constexpr (Q == 19) {
        // pairs (1,2) x, (3,4) y, (5,6) z, (7,8) +x+y, (9,10) +x-y,
        // (11,12) +x+z, (13,14) +x-z, (15,16) +y+z, (17,18) +y-z
        float2 sp[9], d[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            sp[k] = add2(g[2 * k + 1], g[2 * k + 2]);
            d[k] = sub2(g[2 * k + 1], g[2 * k + 2]);
        }
        m = add2(add2(add2(add2(sp[0], sp[1]), add2(sp[2], sp[3])), add2(add2(sp[4], sp[5]), add2(sp[6], sp[7]))),
                 add2(g[0], sp[8]));
        j[0] = add2(add2(add2(d[0], d[3]), add2(d[4], d[5])), d[6]);
        j[1] = sub2(add2(add2(d[1], d[3]), add2(d[7], d[8])), d[4]);
        j[2] = sub2(add2(add2(d[2], d[5]), d[7]), add2(d[6], d[8]));
    } else {
        // D2Q9, Sec. 4.2 numbering: pairs (1,3) x, (2,4) y, (5,7) +x+y, (6,8) -x+y
        const float2 d0 = sub2(g[1], g[3]), d1 = sub2(g[2], g[4]), d2 = sub2(g[5], g[7]), d3 = sub2(g[6], g[8]);
        m = add2(add2(add2(g[1], g[3]), add2(g[2], g[4])), add2(add2(g[5], g[7]), add2(g[6], g[8])));
        m = add2(m, g[0]);
        j[0] = sub2(add2(d0, d2), d3);
        j[1] = add2(add2(d1, d2), d3);
        j[2] = b2(0.f);
    }
}

// Pull direction i of both cells.  SHIFT is the x shift of the direction's
// source (+1: from x - 1, -1: from x + 1, 0: none).
template <typename S, bool REF>
__device__ __forceinline__ float2 pull_dir(const S *__restrict__ in, int src, int shift, const Cols &X,
                                           float ref, float inv)
{
    const S *q = src_row(in, src);
    float2 v;
    if (shift == 0)
        v = Pair<S>::load2(q + X.x0);
    else if (shift > 0)
        v = make_float2(Pair<S>::load1(q + X.pm_a), Pair<S>::load1(q + X.x0));
    else
        v = make_float2(Pair<S>::load1(q + X.pp_a), Pair<S>::load1(q + X.pp_b));
    if constexpr (REF) v = fma2(v, b2(inv), b2(ref));
    return v;
}

template <int Q, typename S>
__device__ __forceinline__ void pull_row2(const S *__restrict__ in, const int src[Q], uint32_t xm,
                                          uint32_t xp, bool xbounce, const Cols &X, const float *dec,
                                          float inv, float2 g[Q])
{
    constexpr bool REF = Storage<S>::kRef;
    if (!xbounce) {
#pragma unroll
        for (int i = 0; i < Q; ++i)
            g[i] = pull_dir<S, REF>(in, src[i], cx<Q>(i), X, REF ? __ldg(dec + i) : 0.f, inv);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int sh = ((xm >> i) & 1u) ? 1 : (((xp >> i) & 1u) ? -1 : 0);
            g[i] = pull_dir<S, REF>(in, src[i], sh, X, REF ? __ldg(dec + i) : 0.f, inv);
        }
    }
}

__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }

__device__ __forceinline__ float2 lagged2(const float *U1, const float *U2, int idx)
{
    return mul2(b2(0.5f), add2(ld2(U1 + idx), ld2(U2 + idx)));
}

__device__ __forceinline__ float2 rcp2(float2 r) { return make_float2(1.f / r.x, 1.f / r.y); }

// Uw1, Uw2 / Us1, Us2: the lagged velocities of the two steps before the
// time level of g (water / solid), as in water_math.
template <int Q>
__device__ __forceinline__ void water_math2(const StepArgs<float> &p, const float *Uw1, const float *Uw2,
                                            const float *Us1, const float *Us2, const RowInfo &R, int x0,
                                            const float2 g[Q], Cell2 &c, float2 j[3])
{
    moments2<Q>(g, c.drho, j);
    c.F[0] = b2(p.G[0]);
    c.F[1] = b2(p.G[1]);
    c.F[2] = b2(p.G[2]);
    const int slot = R.slot;
    if (slot >= 0) {
        const int ns_w = p.n_slots[kFluid], ns_s = p.n_slots[kSolid], nxp = p.nxp;
        const int nface = R.nface;
        for (int a = 0; a < 3; ++a) {
            const float2 uw = lagged2(Uw1, Uw2, (a * ns_w + slot) * nxp + x0);
            float2 f = b2(0.f);
            for (int k = 0; k < nface; ++k) {
                const int q = R.partner[k];
                const float2 de = sub2(uw, lagged2(Us1, Us2, (a * ns_s + q) * nxp + x0));
                const float2 dp = sub2(uw, lagged2(Us1, Us2, ((a + 3) * ns_s + q) * nxp + x0));
                f = sub2(f, fma2(b2(p.g_we), de, mul2(b2(p.g_wp), dp)));
            }
            c.F[a] = add2(c.F[a], f);
        }
    }
    const float2 rinv = rcp2(add2(b2(p.rho0), c.drho));
#pragma unroll
    for (int a = 0; a < 3; ++a) c.u[a] = mul2(fma2(b2(0.5f), c.F[a], j[a]), rinv);
}

template <int Q>
__device__ __forceinline__ void solid_math2(const StepArgs<float> &p, const float *Uw1, const float *Uw2,
                                            const float *Us1, const float *Us2, const RowInfo &R, int x0,
                                            const float2 ge[Q], const float2 gp[Q], Cell2 &ce,
                                            Cell2 &cp, float2 je[3], float2 jp[3])
{
    moments2<Q>(ge, ce.drho, je);
    moments2<Q>(gp, cp.drho, jp);
    float2 Fe[3] = {b2(0.f), b2(0.f), b2(0.f)}, Fp[3] = {b2(0.f), b2(0.f), b2(0.f)};
    const int slot = R.slot;
    if (slot >= 0) {
        const int ns_w = p.n_slots[kFluid], ns_s = p.n_slots[kSolid], nxp = p.nxp;
        const int nface = R.nface;
        for (int a = 0; a < 3; ++a) {
            const float2 ue = lagged2(Us1, Us2, (a * ns_s + slot) * nxp + x0);
            const float2 up = lagged2(Us1, Us2, ((a + 3) * ns_s + slot) * nxp + x0);
            float2 fe = b2(0.f), fp = b2(0.f);
            for (int k = 0; k < nface; ++k) {
                const float2 uw = lagged2(Uw1, Uw2, (a * ns_w + R.partner[k]) * nxp + x0);
                fe = fma2(b2(p.g_we), sub2(uw, ue), fe);
                fp = fma2(b2(p.g_wp), sub2(uw, up), fp);
            }
            Fe[a] = fe;
            Fp[a] = fp;
        }
    }
    // (a + k + se) ue - k up = Je,  -k ue + (b + k + sp) up = Jp.
    const float k = 0.5f * p.g_ep, se = 0.5f * p.g_ec, sp = 0.5f * p.g_pc;
    const float2 A = add2(add2(b2(p.rho0), ce.drho), b2(k + se));
    const float2 B = add2(add2(b2(p.rho0), cp.drho), b2(k + sp));
    const float2 Dinv = rcp2(sub2(mul2(A, B), b2(k * k)));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float2 Je = fma2(b2(0.5f), Fe[a], je[a]);
        const float2 Jp = fma2(b2(0.5f), Fp[a], jp[a]);
        const float2 ue = mul2(fma2(B, Je, mul2(b2(k), Jp)), Dinv);
        const float2 up = mul2(fma2(A, Jp, mul2(b2(k), Je)), Dinv);
        ce.u[a] = ue;
        cp.u[a] = up;
        const float2 d = sub2(ue, up);
        ce.F[a] = sub2(sub2(Fe[a], mul2(b2(p.g_ep), d)), mul2(b2(p.g_ec), ue));
        cp.F[a] = sub2(fma2(b2(p.g_ep), d, Fp[a]), mul2(b2(p.g_pc), up));
    }
}

// Unbiased rounding of the FP32 fix-up (FP32 storage).  The fix-up's
// increments are mostly below half an ulp of the populations they go to
// (about 1e-10 against |g| ~ 2e-3), so round-to-nearest drops them, and in
// a steady state it drops them the same way in every step: a per-row bias
// of the stored momentum that the slowest shear mode accumulates (velocity
// error ~4e-6 after 10^4 steps on the benchmark pipe).  Here each increment
// is added with a uniform dither of one ulp of the target, a + RN(b + d),
// d in [-ulp/2, ulp/2): the rounded sum is a + b on average (subtractive-free
// dither), and the dither changes from row to row and step to step.  The
// bits come from the lowbias32 integer hash (C. Wellons) of the row's
// cross-section cell, the species and the step: every cell of a row gets
// the same dither, so that a state that does not vary along x stays so
// (and a lattice reproduces its x-slices), while the bias, which a
// steady state repeats step after step, becomes noise in time.
__device__ __forceinline__ uint32_t lowbias32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Uniform in [-1/2, 1/2) from the top 23 bits of r.
__device__ __forceinline__ float dither_unit(uint32_t r) { return __int_as_float(0x3f800000u | (r >> 9)) - 1.5f; }

// One ulp of a normal a (exponent field times 2^-23; 0 for zero or a subnormal).
__device__ __forceinline__ float ulp_of(float a)
{
    return __int_as_float(__float_as_int(a) & 0x7f800000) * 1.1920928955078125e-7f;
}

// a + b with a one-ulp dither (r: random bits; the same dither fraction for
// both cells, each scaled by its own ulp).
__device__ __forceinline__ float2 add2_dither(float2 a, float2 b, uint32_t r)
{
    const float u = dither_unit(r);
    return add2(a, add2(b, make_float2(u * ulp_of(a.x), u * ulp_of(a.y))));
}

// Dither seed of the row with cross-section cell cs for species s at step n.
__device__ __forceinline__ uint32_t dither_seed(uint32_t cs, uint32_t n, int s)
{
    return lowbias32(cs ^ lowbias32(n * 3u + (uint32_t)s));
}

// BGK + Guo collision of both cells, per pair of opposite directions, then
// the FP32 fix-up of mass and momentum (see collide; q as there: 1 for the
// second-order equilibrium, 0 for the linear one of phonons as damped
// waves).  g is left holding g*.
//
// DITHER (FP32 storage): the residuals of the fix-up are summed from the
// per-direction differences g_i - g*_i, which are small, so that they are
// exact to about 1e-12 (the sums Sum g_i and Sum g*_i of the plain fix-up
// each round at the scale of |g|), and the increments are added with
// add2_dither (seed sd: dither_seed).  16-bit storage rounds the stored
// differences to nearest anyway and keeps the plain fix-up.
template <int Q, bool FIX = true, bool DITHER = false>
__device__ __forceinline__ void collide2(float2 g[Q], const Cell2 &c, const float2 j[3], float rho0,
                                         float om, float q = 1.f, uint32_t sd = 0u)
{
    const float2 rho = add2(b2(rho0), c.drho);
    const float2 uu = fma2(c.u[2], c.u[2], fma2(c.u[1], c.u[1], mul2(c.u[0], c.u[0])));
    const float2 uF = fma2(c.u[2], c.F[2], fma2(c.u[1], c.F[1], mul2(c.u[0], c.F[0])));
    const float2 e0 = fma2(mul2(b2(-1.5f * q), rho), uu, c.drho);
    const float2 r45 = mul2(b2(4.5f * q), rho);
    const float2 m3uF = mul2(b2(-3.f * q), uF);
    const float om1 = 1.f - om, fo = 1.f - 0.5f * om;
    constexpr bool DIFF = FIX && DITHER;
    float2 dm = b2(0.f), dj[3] = {b2(0.f), b2(0.f), b2(0.f)};  // Sum (g - g*), Sum c (g - g*)
    {
        const float w = float(wt<Q>(0));
        const float2 g0 = g[0];
        g[0] = fma2(b2(om1), g[0], fma2(b2(om * w), e0, mul2(b2(fo * w), m3uF)));
        if constexpr (DIFF) dm = sub2(g0, g[0]);
    }
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (opp<Q>(i) < i) continue;
        const int ib = opp<Q>(i);
        const float w = float(wt<Q>(i));
        const float2 cu = cdot2<Q>(i, c.u);
        const float2 cF = cdot2<Q>(i, c.F);
        // even parts: e0 + 4.5 rho cu^2 and -3 u.F + 9 cu cF
        const float2 se = fma2(r45, mul2(cu, cu), e0);
        const float2 sf = fma2(b2(9.f * q), mul2(cu, cF), m3uF);
        const float2 S = fma2(b2(om * w), se, mul2(b2(fo * w), sf));
        // odd parts: 3 rho cu and 3 cF
        const float2 A = fma2(mul2(b2(3.f * om * w), rho), cu, mul2(b2(3.f * fo * w), cF));
        const float2 gi = g[i], gb = g[ib];
        g[i] = fma2(b2(om1), gi, add2(S, A));
        g[ib] = fma2(b2(om1), gb, sub2(S, A));
        if constexpr (DIFF) {
            const float2 di = sub2(gi, g[i]), db = sub2(gb, g[ib]);
            dm = add2(dm, add2(di, db));
            const float2 dd = sub2(di, db);
            const int cc[3] = {cx<Q>(i), cy<Q>(i), cz<Q>(i)};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (cc[k] > 0) dj[k] = add2(dj[k], dd);
                if (cc[k] < 0) dj[k] = sub2(dj[k], dd);
            }
        }
    }
    if constexpr (!FIX) return;
    if constexpr (DIFF) {
        // Sum g*_final = Sum g and Sum c g*_final = Sum c g + F
        g[0] = add2_dither(g[0], dm, sd);
#pragma unroll
        for (int k = 0; k < (Q == 19 ? 3 : 2); ++k) {
            const float2 h = mul2(b2(0.5f), add2(dj[k], c.F[k]));
            const int ip = dir_index<Q>(k == 0, k == 1, k == 2);
            const int im = dir_index<Q>(-(k == 0), -(k == 1), -(k == 2));
            const uint32_t mp = 0x9E3779B9u * (uint32_t)(2 * k + 1) | 1u, mm = 0x9E3779B9u * (uint32_t)(2 * k + 2) | 1u;
            g[ip] = add2_dither(g[ip], h, sd * mp);
            g[im] = add2_dither(g[im], make_float2(-h.x, -h.y), sd * mm);
        }
        return;
    }
    float2 m, pm[3];
    moments2<Q>(g, m, pm);
    const float2 px = pm[0], py = pm[1];
    g[0] = add2(g[0], sub2(c.drho, m));
    const float2 hx = mul2(b2(0.5f), add2(sub2(j[0], px), c.F[0]));
    const float2 hy = mul2(b2(0.5f), add2(sub2(j[1], py), c.F[1]));
    g[dir_index<Q>(1, 0, 0)] = add2(g[dir_index<Q>(1, 0, 0)], hx);
    g[dir_index<Q>(-1, 0, 0)] = sub2(g[dir_index<Q>(-1, 0, 0)], hx);
    g[dir_index<Q>(0, 1, 0)] = add2(g[dir_index<Q>(0, 1, 0)], hy);
    g[dir_index<Q>(0, -1, 0)] = sub2(g[dir_index<Q>(0, -1, 0)], hy);
    if (Q == 19) {
        const float2 pz = pm[2];
        const float2 hz = mul2(b2(0.5f), add2(sub2(j[2], pz), c.F[2]));
        g[dir_index<Q>(0, 0, 1)] = add2(g[dir_index<Q>(0, 0, 1)], hz);
        g[dir_index<Q>(0, 0, -1)] = sub2(g[dir_index<Q>(0, 0, -1)], hz);
    }
}

// Store g* of both cells, encoded against the row's references for 16-bit
// storage: (g - ref) * scale = fma(g, scale, -ref * scale) exactly, scale
// being a power of two.  The second cell of an odd row's last pair goes to
// the row padding, which nothing reads (one store per direction, no
// predicated pair).
template <int Q, typename S>
__device__ __forceinline__ void store_pair(const float2 g[Q], S *__restrict__ out, int row_stride,
                                           int base, const float *enc, float scale)
{
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float2 v = g[i];
        if constexpr (Storage<S>::kRef) v = fma2(v, b2(scale), b2(-__ldg(enc + i) * scale));
        Pair<S>::store2(out + (long long)i * row_stride + base, v);
    }
}

__device__ __forceinline__ void store_u2(float *q, float2 v) { *reinterpret_cast<float2 *>(q) = v; }

// x-sums over the 32-wide segments of a warp whose threads hold CPT cells
// each (32 / CPT threads per segment) of NV per-thread values (the sums of
// their live cells), written by the first thread of each segment to
// acc + seg * 2Q; a segment past the end of the row (seg < 0) is skipped.
template <int CPT, int NV>
__device__ __forceinline__ void segment_xsum(const float (&v)[NV], float *acc, int seg, int stride)
{
    constexpr int L = 32 / CPT;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        float s = v[k];
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((lane & (L - 1)) == 0 && seg >= 0) acc[(size_t)seg * stride + k] = s;
    }
}

// Segment of the calling thread's cells: the warp's first x plus 32 per
// segment, or -1 past the end of the row.
template <int CPT>
__device__ __forceinline__ int thread_segment(const StepArgs<float> &p, bool water, int row, int x_first)
{
    const int lane = threadIdx.x & 31;
    const int xs = x_first - CPT * lane + 32 * (lane / (32 / CPT));  // first x of the segment
    if (xs >= p.nx) return -1;
    return (water ? 0 : p.nseg_w) + row * p.nch32 + xs / 32;
}

template <int Q, typename S, bool ACC, bool NOISE = false>
__device__ __forceinline__ void step_body2(const StepArgs<float> &p, int b)
{
    // solid blocks (two species each, the heavier work) first, so that the
    // grid's last wave holds the lighter water blocks
    const int nsb = p.n_rows[kSolid] * p.snchunk_s;
    const bool water = b >= nsb;
    const int bb = water ? b - nsb : b;
    const int nch = water ? p.snchunk_w : p.snchunk_s;
    int row = bb / nch;
    const int xt = (bb - row * nch) * blockDim.x + threadIdx.x;
    const int x_first = 2 * xt;
    bool live = x_first < p.nx;
    if constexpr (KLB_BOUNDS) {
        if (live && !row_indices_ok<Q>(p, water, row, 0, x_first + 1)) {
            live = false;
            row = 0;
        }
    }
    if constexpr (!ACC) {
        if (!live) return;  // no warp-wide operation follows
    }
    Cols X;
    X.x0 = live ? x_first : 0;  // a dead thread of an accumulating pass computes cells 0, 1
    const bool both = X.x0 + 1 < p.nx && live;
    X.pm_a = X.x0 == 0 ? p.nx - 1 : X.x0 - 1;
    X.pp_a = X.x0 + 1 >= p.nx ? 0 : X.x0 + 1;
    X.pp_b = X.x0 + 2 >= p.nx ? 0 : X.x0 + 2;
    const int nxp = p.nxp;
    const float inv = p.inv_scale, sc = p.scale;

    const RowInfo &R = p.rows[water ? kFluid : kSolid][row];
    const int4 *t4 = reinterpret_cast<const int4 *>(&R);
    int src[20];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        const int4 q = __ldg(t4 + v);
        src[4 * v] = q.x;
        src[4 * v + 1] = q.y;
        src[4 * v + 2] = q.z;
        src[4 * v + 3] = q.w;
    }
    const uint32_t xm = (uint32_t)src[19];
    const int4 q5 = __ldg(t4 + 5);  // xp, slot, nface, partner[0]
    const int4 q7 = __ldg(t4 + 7);  // flags, cs
    const uint32_t xp = (uint32_t)q5.x;
    const bool xbounce = (q7.x & kXBounce) != 0;

    const int seg = ACC ? thread_segment<2>(p, water, row, x_first) : -1;
    pdl_wait();  // populations, lagged velocities, references and the period count below
    constexpr bool DITHER = !Storage<S>::kRef;
    const uint32_t n_step = p.step_lo + (p.step_reps ? *p.step_reps * (uint32_t)p.step_period : 0u);

    if (water) {
        float2 g[Q], j[3];
        Cell2 c;
        pull_row2<Q, S>(static_cast<const S *>(p.in[0]), src, xm, xp, xbounce, X,
                        ref_row<float, S>(p.dec_in[0], row), inv, g);
        water_math2<Q>(p, p.U1[kFluid], p.U2[kFluid], p.U1[kSolid], p.U2[kSolid], R, X.x0, g, c, j);
        if (q5.y >= 0 && live) {
            const int ns = p.n_slots[kFluid];
            for (int a = 0; a < 3; ++a) store_u2(p.U0[kFluid] + (a * ns + q5.y) * nxp + X.x0, c.u[a]);
        }
        collide2<Q, true, DITHER>(g, c, j, p.rho0, p.om[0], 1.f, dither_seed((uint32_t)q7.y, n_step, 0));
        if constexpr (NOISE) {
            const uint32_t cell = (uint32_t)X.x0 + (uint32_t)p.nx * (uint32_t)q7.y;
            thermal_noise<Q, float>(p, cell, [&](int i, float v) { g[i].x += v; });
            if (both) thermal_noise<Q, float>(p, cell + 1, [&](int i, float v) { g[i].y += v; });
        }
        if (live)
            store_pair<Q, S>(g, static_cast<S *>(p.out[0]), p.n_rows[kFluid] * nxp, row * nxp + X.x0,
                             ref_row<float, S>(p.enc_out[0], row), sc);
        if constexpr (ACC) {
            float acc[2 * Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                acc[i] = (live ? g[i].x : 0.f) + (both ? g[i].y : 0.f);
                acc[Q + i] = 0.f;
            }
            segment_xsum<2, 2 * Q>(acc, p.acc, seg, 2 * Q);
        }
        return;
    }

    float2 ge[Q], gp[Q], je[3], jp[3];
    Cell2 ce, cp;
    pull_row2<Q, S>(static_cast<const S *>(p.in[1]), src, xm, xp, xbounce, X,
                    ref_row<float, S>(p.dec_in[1], row), inv, ge);
    pull_row2<Q, S>(static_cast<const S *>(p.in[2]), src, xm, xp, xbounce, X,
                    ref_row<float, S>(p.dec_in[2], row), inv, gp);
    solid_math2<Q>(p, p.U1[kFluid], p.U2[kFluid], p.U1[kSolid], p.U2[kSolid], R, X.x0, ge, gp, ce, cp, je, jp);
    if (q5.y >= 0 && live) {
        const int ns = p.n_slots[kSolid];
        for (int a = 0; a < 3; ++a) {
            store_u2(p.U0[kSolid] + (a * ns + q5.y) * nxp + X.x0, ce.u[a]);
            store_u2(p.U0[kSolid] + ((a + 3) * ns + q5.y) * nxp + X.x0, cp.u[a]);
        }
    }
    const int stride = p.n_rows[kSolid] * nxp, base = row * nxp + X.x0;
    collide2<Q, true, DITHER>(ge, ce, je, p.rho0, p.om[1], 1.f, dither_seed((uint32_t)q7.y, n_step, 1));
    if (live)
        store_pair<Q, S>(ge, static_cast<S *>(p.out[1]), stride, base, ref_row<float, S>(p.enc_out[1], row), sc);
    float acc[ACC ? 2 * Q : 1];
    if constexpr (ACC) {
#pragma unroll
        for (int i = 0; i < Q; ++i) acc[i] = (live ? ge[i].x : 0.f) + (both ? ge[i].y : 0.f);
    }
    pull_row2<Q, S>(static_cast<const S *>(p.in[2]), src, xm, xp, xbounce, X,
                    ref_row<float, S>(p.dec_in[2], row), inv, gp);
    collide2<Q, true, DITHER>(gp, cp, jp, p.rho0, p.om[2], p.q_p, dither_seed((uint32_t)q7.y, n_step, 2));
    if (live)
        store_pair<Q, S>(gp, static_cast<S *>(p.out[2]), stride, base, ref_row<float, S>(p.enc_out[2], row), sc);
    if constexpr (ACC) {
#pragma unroll
        for (int i = 0; i < Q; ++i) acc[Q + i] = (live ? gp[i].x : 0.f) + (both ? gp[i].y : 0.f);
        segment_xsum<2, 2 * Q>(acc, p.acc, seg, 2 * Q);
    }
}

// Observation pass with two cells per thread (FP32 arithmetic), on the step
// kernel's grid (solid blocks first): the velocities of the current step
// (lagged velocities U1, U2) and, for the residual, of the previous one (U2,
// U3), from the same pulls and arithmetic as the step, reduced per block in
// FP64 into the partial sums of the observation (observe_reduce_store).
__device__ __forceinline__ bool finite2(const Cell2 &c, int e)
{
    const float v[4] = {e ? c.drho.y : c.drho.x, e ? c.u[0].y : c.u[0].x, e ? c.u[1].y : c.u[1].x,
                        e ? c.u[2].y : c.u[2].x};
    return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]) && isfinite(v[3]);
}

template <int Q, typename S>
__global__ void __launch_bounds__(kBlockX, 4) k_observe2(const StepArgs<float> p)
{
    const int b = blockIdx.x;
    const int nsb = p.n_rows[kSolid] * p.snchunk_s;
    const bool water = b >= nsb;
    const int bb = water ? b - nsb : b;
    const int nch = water ? p.snchunk_w : p.snchunk_s;
    int row = bb / nch;
    const int x_first = 2 * ((bb - row * nch) * (int)blockDim.x + (int)threadIdx.x);
    bool live = x_first < p.nx;
    if constexpr (KLB_BOUNDS) {
        if (live && !row_indices_ok<Q>(p, water, row, 0, x_first + 1)) {
            live = false;
            row = 0;
        }
    }
    const bool both = live && x_first + 1 < p.nx;
    double s[kNumSums];
#pragma unroll
    for (int k = 0; k < kNumSums; ++k) s[k] = 0.0;
    const RowInfo &R = p.rows[water ? kFluid : kSolid][row];
    if (live) {
        Cols X;
        X.x0 = x_first;
        X.pm_a = X.x0 == 0 ? p.nx - 1 : X.x0 - 1;
        X.pp_a = X.x0 + 1 >= p.nx ? 0 : X.x0 + 1;
        X.pp_b = X.x0 + 2 >= p.nx ? 0 : X.x0 + 2;
        const float inv = p.inv_scale;
        const int4 *t4 = reinterpret_cast<const int4 *>(&R);
        int src[20];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const int4 q = __ldg(t4 + v);
            src[4 * v] = q.x;
            src[4 * v + 1] = q.y;
            src[4 * v + 2] = q.z;
            src[4 * v + 3] = q.w;
        }
        const uint32_t xm = (uint32_t)src[19];
        const int4 q5 = __ldg(t4 + 5);
        const int4 q7 = __ldg(t4 + 7);
        const uint32_t xp = (uint32_t)q5.x;
        const bool xbounce = (q7.x & kXBounce) != 0;
        // the previous step first (for the residual), keeping only its u_x,
        // so that the current step's values and sums are live alone
        if (water) {
            float2 g[Q], j[3];
            float2 uq = b2(0.f);
            if (p.residual_valid) {
                Cell2 cq;
                pull_row2<Q, S>(static_cast<const S *>(p.in_prev[0]), src, xm, xp, xbounce, X,
                                ref_row<float, S>(p.dec_prev[0], row), inv, g);
                water_math2<Q>(p, p.U2[kFluid], p.U3[kFluid], p.U2[kSolid], p.U3[kSolid], R, X.x0, g, cq, j);
                uq = cq.u[0];
            }
            Cell2 c;
            pull_row2<Q, S>(static_cast<const S *>(p.in[0]), src, xm, xp, xbounce, X,
                            ref_row<float, S>(p.dec_in[0], row), inv, g);
            water_math2<Q>(p, p.U1[kFluid], p.U2[kFluid], p.U1[kSolid], p.U2[kSolid], R, X.x0, g, c, j);
            const double u0 = c.u[0].x, u1 = both ? (double)c.u[0].y : 0.0;
            s[kSumUxFluid] = u0 + u1;
            // the second cell of an odd row's last pair lies in the padding:
            // none of its values enters a sum
            s[kSumMomW] = (double)(p.rho0 + c.drho.x) * u0 + (both ? (double)(p.rho0 + c.drho.y) * u1 : 0.0);
            s[kSumMassW] = (double)c.drho.x + (both ? (double)c.drho.y : 0.0);
            s[kSumNonfinite] = (finite2(c, 0) ? 0.0 : 1.0) + (both && !finite2(c, 1) ? 1.0 : 0.0);
            const S *in0 = static_cast<const S *>(p.in[0]);
            s[kSumClipped] = (clipped_cell<Q, S>(in0, R, X.x0, X.pm_a, X.pp_a) ? 1.0 : 0.0) +
                             (both && clipped_cell<Q, S>(in0, R, X.x0 + 1, X.x0, X.pp_b) ? 1.0 : 0.0);
            if (R.flags & kFitRow) s[kSumFitUD2] = (u0 + u1) * (double)R.d2;
            if (p.residual_valid)
                s[kSumResidual] = fmax(fabs(u0 - (double)uq.x), both ? fabs(u1 - (double)uq.y) : 0.0);
        } else {
            float2 ge[Q], gp[Q], je[3], jp[3];
            float2 eq = b2(0.f), pq = b2(0.f);
            if (p.residual_valid) {
                Cell2 qe, qp;
                pull_row2<Q, S>(static_cast<const S *>(p.in_prev[1]), src, xm, xp, xbounce, X,
                                ref_row<float, S>(p.dec_prev[1], row), inv, ge);
                pull_row2<Q, S>(static_cast<const S *>(p.in_prev[2]), src, xm, xp, xbounce, X,
                                ref_row<float, S>(p.dec_prev[2], row), inv, gp);
                solid_math2<Q>(p, p.U2[kFluid], p.U3[kFluid], p.U2[kSolid], p.U3[kSolid], R, X.x0, ge, gp, qe, qp,
                               je, jp);
                eq = qe.u[0];
                pq = qp.u[0];
            }
            Cell2 ce, cp;
            pull_row2<Q, S>(static_cast<const S *>(p.in[1]), src, xm, xp, xbounce, X,
                            ref_row<float, S>(p.dec_in[1], row), inv, ge);
            pull_row2<Q, S>(static_cast<const S *>(p.in[2]), src, xm, xp, xbounce, X,
                            ref_row<float, S>(p.dec_in[2], row), inv, gp);
            solid_math2<Q>(p, p.U1[kFluid], p.U2[kFluid], p.U1[kSolid], p.U2[kSolid], R, X.x0, ge, gp, ce, cp, je,
                           jp);
            const double e0 = ce.u[0].x, e1 = both ? (double)ce.u[0].y : 0.0;
            const double p0 = cp.u[0].x, p1 = both ? (double)cp.u[0].y : 0.0;
            s[kSumUxE] = e0 + e1;
            s[kSumUxP] = p0 + p1;
            s[kSumMomE] = (double)(p.rho0 + ce.drho.x) * e0 + (both ? (double)(p.rho0 + ce.drho.y) * e1 : 0.0);
            s[kSumMomP] = (double)(p.rho0 + cp.drho.x) * p0 + (both ? (double)(p.rho0 + cp.drho.y) * p1 : 0.0);
            s[kSumMassE] = (double)ce.drho.x + (both ? (double)ce.drho.y : 0.0);
            s[kSumMassP] = (double)cp.drho.x + (both ? (double)cp.drho.y : 0.0);
            s[kSumNonfinite] = (finite2(ce, 0) ? 0.0 : 1.0) + (finite2(cp, 0) ? 0.0 : 1.0) +
                               (both && !finite2(ce, 1) ? 1.0 : 0.0) + (both && !finite2(cp, 1) ? 1.0 : 0.0);
            const S *in1 = static_cast<const S *>(p.in[1]), *in2 = static_cast<const S *>(p.in[2]);
            s[kSumClipped] = (clipped_cell<Q, S>(in1, R, X.x0, X.pm_a, X.pp_a) ? 1.0 : 0.0) +
                             (clipped_cell<Q, S>(in2, R, X.x0, X.pm_a, X.pp_a) ? 1.0 : 0.0) +
                             (both && clipped_cell<Q, S>(in1, R, X.x0 + 1, X.x0, X.pp_b) ? 1.0 : 0.0) +
                             (both && clipped_cell<Q, S>(in2, R, X.x0 + 1, X.x0, X.pp_b) ? 1.0 : 0.0);
            if (p.residual_valid) {
                double r = fmax(fabs(e0 - (double)eq.x), fabs(p0 - (double)pq.x));
                if (both) r = fmax(r, fmax(fabs(e1 - (double)eq.y), fabs(p1 - (double)pq.y)));
                s[kSumResidual] = r;
            }
        }
    }
    observe_reduce_store(s, water, water ? R.flags : 0, (double)R.d2, live ? (both ? 2 : 1) : 0,
                         p.partials + (size_t)b * kNumSums);
}

}  // namespace klb
