// CUDA kernels of the KLB step for sm_103a (templates; instantiated per
// lattice in klb_kernels_q9.cu and klb_kernels_q19.cu).
//
// One fused kernel per lattice step (k_step) updates all three species
// (Sec. 4: one population set per species, {h_i, e_i, p_i}):
//   pull-stream (boundary rules of Sec. 4.2, precomputed per row) ->
//   moments -> interface friction (Eq. 27) from lagged velocities ->
//   trapezoidal electron-phonon friction and crystal sinks (Eqs. 12, 13, 16) ->
//   Guo velocity -> BGK collision with Guo forcing (body force of Eq. 2) ->
//   store (A-B: the state is read from one buffer and written to the other).
//
// Layout: structure of arrays, per species [direction][row][x] with rows of
// nxp elements (x fastest, rows padded to 32 elements), so every load and
// store of a warp is a contiguous run of x.  A block covers up to 128
// consecutive x of one row; the row table (sources, x shifts, interface
// partners) is block-uniform.  A solid block updates the electrons and
// phonons of its row together; the step grid puts the solid blocks first
// (the heavier work, so that its last wave holds water blocks), the
// observation, field and initialisation grids the water blocks first.
//
// Template parameters: Q (9 or 19), T the arithmetic type (double or float)
// and S the storage type of the populations (T itself, or __half /
// __nv_bfloat16 with FP32 arithmetic).  Reduced-precision storage keeps, per
// row and direction, the difference from an FP32 reference population (the
// row's x-average, refreshed every few steps), times a fixed power of two:
//   stored = S((g - ref[row][i]) * scale),  g = float(stored) / scale + ref.
// The reference of a pulled population is that of its source row (table
// `dec`), the reference of a stored one that of its own row (table `enc`).
//
// k_lattice runs the same per-cell arithmetic for the observation pass
// (velocities of the current and previous step reduced in FP64) and the
// field pass; k_init starts from local equilibria.

#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstddef>

#include "klb_internal.h"

#ifndef KLB_BOUNDS
#define KLB_BOUNDS 0
#endif

namespace klb {

// ---------------------------------------------------------------------------
// Lattice constants, folded at compile time inside unrolled loops.

template <int Q> __host__ __device__ constexpr int cx(int i);
template <int Q> __host__ __device__ constexpr int cy(int i);
template <int Q> __host__ __device__ constexpr int cz(int i);
template <int Q> __host__ __device__ constexpr double wt(int i);

template <> __host__ __device__ constexpr int cx<9>(int i)
{
    return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
template <> __host__ __device__ constexpr int cy<9>(int i)
{
    return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
template <> __host__ __device__ constexpr int cz<9>(int) { return 0; }
template <> __host__ __device__ constexpr double wt<9>(int i)
{
    return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// D3Q19: 0 rest; 1..6 (+x,-x,+y,-y,+z,-z); 7..18 edges in opposite pairs.
__host__ __device__ constexpr int c19(int i, int a)
{
    constexpr int t[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                              {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                              {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                              {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    return t[i][a];
}
template <> __host__ __device__ constexpr int cx<19>(int i) { return c19(i, 0); }
template <> __host__ __device__ constexpr int cy<19>(int i) { return c19(i, 1); }
template <> __host__ __device__ constexpr int cz<19>(int i) { return c19(i, 2); }
template <> __host__ __device__ constexpr double wt<19>(int i)
{
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// ---------------------------------------------------------------------------
// Storage types.

template <typename S> struct Storage;
template <> struct Storage<float> {
    static constexpr bool kRef = false;
    __device__ static float load(const float *p) { return __ldg(p); }
    __device__ static void store(float *p, float v) { *p = v; }
};
template <> struct Storage<double> {
    static constexpr bool kRef = false;
    __device__ static double load(const double *p) { return __ldg(p); }
    __device__ static void store(double *p, double v) { *p = v; }
};
// 16-bit encodes round to nearest and saturate: a value beyond the largest
// finite magnitude is stored as that magnitude (not as infinity), which the
// observation pass counts (clipped_cell); NaN stays NaN.
__device__ __forceinline__ unsigned short f32_to_f16_sat(float v)
{
    unsigned short r;
    asm("cvt.rn.satfinite.f16.f32 %0, %1;" : "=h"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ unsigned short f32_to_bf16_sat(float v)
{
    unsigned short r;
    asm("cvt.rn.satfinite.bf16.f32 %0, %1;" : "=h"(r) : "f"(v));
    return r;
}
// Pairs: the low half holds v.x, the high half v.y.
__device__ __forceinline__ unsigned f32x2_to_f16x2_sat(float2 v)
{
    unsigned r;
    asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(v.y), "f"(v.x));
    return r;
}
__device__ __forceinline__ unsigned f32x2_to_bf16x2_sat(float2 v)
{
    unsigned r;
    asm("cvt.rn.satfinite.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(v.y), "f"(v.x));
    return r;
}

template <> struct Storage<__half> {
    static constexpr bool kRef = true;
    static constexpr unsigned short kMaxBits = 0x7bffu;  // 65504
    __device__ static float load(const __half *p)
    {
        return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static void store(__half *p, float v)
    {
        *reinterpret_cast<unsigned short *>(p) = f32_to_f16_sat(v);
    }
};
template <> struct Storage<__nv_bfloat16> {
    static constexpr bool kRef = true;
    static constexpr unsigned short kMaxBits = 0x7f7fu;  // 3.3895e38
    __device__ static float load(const __nv_bfloat16 *p)
    {
        return __bfloat162float(
            __ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static void store(__nv_bfloat16 *p, float v)
    {
        *reinterpret_cast<unsigned short *>(p) = f32_to_bf16_sat(v);
    }
};

// Whether any of the Q pulled 16-bit populations of a cell sits at the
// largest finite magnitude (a saturated encode); false for wider storage.
template <int Q, typename S>
__device__ __forceinline__ bool clipped_cell(const S *__restrict__ in, const RowInfo &R, int x, int xm1, int xp1)
{
    if constexpr (!Storage<S>::kRef) {
        return false;
    } else {
        bool any = false;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int xs = ((R.xm >> i) & 1u) ? xm1 : (((R.xp >> i) & 1u) ? xp1 : x);
            const unsigned short b =
                __ldg(reinterpret_cast<const unsigned short *>(in + (long long)R.src[i] * kRowAlign + xs));
            any |= (b & 0x7fffu) == Storage<S>::kMaxBits;
        }
        return any;
    }
}

// ---------------------------------------------------------------------------

template <typename T>
struct Cell {
    T drho;   // density deviation
    T u[3];   // Guo velocity (j + F/2) / rho
    T F[3];   // total force density
};

// c_i . v with only the non-zero velocity components (no additions of 0,
// which IEEE signed zeros keep the compiler from dropping).
template <int Q, typename T>
__device__ __forceinline__ T cdot(int i, const T v[3])
{
    const int c[3] = {cx<Q>(i), cy<Q>(i), cz<Q>(i)};
    T r = T(0);
    bool any = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (c[a] == 0) continue;
        if (!any)
            r = c[a] > 0 ? v[a] : -v[a];
        else
            r = c[a] > 0 ? r + v[a] : r - v[a];
        any = true;
    }
    return r;
}

// Sum of +-g_i over the directions with c_ia = +-1 (first term not added to 0).
template <int Q, typename T>
__device__ __forceinline__ T cmoment(int a, const T g[Q])
{
    T r = T(0);
    bool any = false;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int c = a == 0 ? cx<Q>(i) : (a == 1 ? cy<Q>(i) : cz<Q>(i));
        if (c == 0) continue;
        if (!any)
            r = c > 0 ? g[i] : -g[i];
        else
            r = c > 0 ? r + g[i] : r - g[i];
        any = true;
    }
    return r;
}

template <int Q, typename T>
__device__ __forceinline__ void moments(const T g[Q], T &drho, T j[3])
{
    drho = g[0];
#pragma unroll
    for (int i = 1; i < Q; ++i) drho += g[i];
    j[0] = cmoment<Q, T>(0, g);
    j[1] = cmoment<Q, T>(1, g);
    j[2] = Q == 19 ? cmoment<Q, T>(2, g) : T(0);
}

// Index of the direction with velocity (a, b, c), at compile time.
template <int Q>
__host__ __device__ constexpr int dir_index(int a, int b, int c)
{
    int k = -1;
    for (int i = 0; i < Q; ++i)
        if (cx<Q>(i) == a && cy<Q>(i) == b && cz<Q>(i) == c) k = i;
    return k;
}

// Reference rows of reduced-precision storage: kRefStride floats per row.
template <typename T, typename S>
__device__ __forceinline__ const float *ref_row(const float *table, int row)
{
    return Storage<S>::kRef ? table + (size_t)row * kRefStride : nullptr;
}

// BGK with Guo forcing, deviation form:
// g*_i = g_i + om (geq_i - g_i) + (1 - om/2) w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F,
// geq_i = w_i [drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)].
// q scales every term of second order in u (and the matching u.F, (c.u)(c.F)
// terms of the source): q = 1 is the scheme above (multiplying by 1 and 9 * 1
// is exact, so its results do not change); q = 0 gives the linear equilibrium
// w_i [drho + 3 rho c.u] and source (1 - om/2) w_i 3 c.F of phonons as the
// damped linear waves of Sec. 3.4.
// The exact scheme conserves mass and gives post-collision momentum j + F.
// In FP32 the lattice weights (1/18, 1/36, ...) are not representable, and
// the rounded weights bias both moments by the same relative amount in every
// cell and every step, a drift that accumulates over the slow relaxation of
// the channel flow.  FP32 therefore restores the two moments after the
// collision: the mass residual goes to the rest population, the momentum
// residual of each axis to its pair of axis populations.  The momentum
// residual is formed as (j - p) + F, not (j + F) - p: j and p differ by about
// F, so j - p is exact and F is added to a small number.  Rounding j + F
// instead would put a systematic error on the state: j is a multiple of its
// own ulp and F changes little from step to step, so RN(j + F) - (j + F)
// repeats with the same sign in every cell of a plug flow and every step
// (for u in [2^-8, 2^-7) and F = 1e-6 it is -0.48 ulp(j), -2.2e-4 F; the
// velocity drifts by that fraction of the drive).  The remaining rounding is
// unbiased.  g is left holding g*.
template <int Q, typename T>
__device__ __forceinline__ void collide(T g[Q], const Cell<T> &c, const T j[3], T rho0, T om, T q = T(1))
{
    const T rho = rho0 + c.drho;
    const T uu = c.u[0] * c.u[0] + c.u[1] * c.u[1] + c.u[2] * c.u[2];
    const T uF = c.u[0] * c.F[0] + c.u[1] * c.F[1] + c.u[2] * c.F[2];
    const T e0 = c.drho - (T(1.5) * q) * rho * uu;
    const T r3 = T(3) * rho, r45 = (T(4.5) * q) * rho;
    const T m3uF = (T(-3) * q) * uF;
    const T om1 = T(1) - om;
    const T fo = T(1) - T(0.5) * om;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T w = T(wt<Q>(i));
        if (i == 0) {  // rest population: c = 0
            g[0] = om1 * g[0] + (om * w) * e0 + (fo * w) * m3uF;
            continue;
        }
        const T cu = cdot<Q, T>(i, c.u);
        const T cF = cdot<Q, T>(i, c.F);
        const T teq = e0 + cu * (r3 + r45 * cu);
        const T tF = m3uF + cF * (T(3) + (T(9) * q) * cu);
        g[i] = om1 * g[i] + (om * w) * teq + (fo * w) * tF;
    }
    if (sizeof(T) == 4) {
        T m = g[0];
#pragma unroll
        for (int i = 1; i < Q; ++i) m += g[i];
        const T p[3] = {cmoment<Q, T>(0, g), cmoment<Q, T>(1, g),
                        Q == 19 ? cmoment<Q, T>(2, g) : T(0)};
        g[0] += c.drho - m;
        const T hx = T(0.5) * ((j[0] - p[0]) + c.F[0]);
        const T hy = T(0.5) * ((j[1] - p[1]) + c.F[1]);
        g[dir_index<Q>(1, 0, 0)] += hx;
        g[dir_index<Q>(-1, 0, 0)] -= hx;
        g[dir_index<Q>(0, 1, 0)] += hy;
        g[dir_index<Q>(0, -1, 0)] -= hy;
        if (Q == 19) {
            const T hz = T(0.5) * ((j[2] - p[2]) + c.F[2]);
            g[dir_index<Q>(0, 0, 1)] += hz;
            g[dir_index<Q>(0, 0, -1)] -= hz;
        }
    }
}

// Store g* of one cell: out[i * row_stride + base] (64-bit plane offsets), encoded against the
// row's references `enc` for reduced-precision storage.
template <int Q, typename T, typename S>
__device__ __forceinline__ void store_cell(const T g[Q], S *__restrict__ out, int row_stride,
                                           int base, const float *enc, float scale)
{
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if constexpr (Storage<S>::kRef)
            Storage<S>::store(out + (long long)i * row_stride + base, (float(g[i]) - __ldg(enc + i)) * scale);
        else
            Storage<S>::store(out + (long long)i * row_stride + base, g[i]);
    }
}

// First element of the source row of a RowInfo::src entry (kRowAlign units:
// the product is 64-bit, so class buffers may exceed 2^31 elements).
template <typename S>
__device__ __forceinline__ const S *src_row(const S *in, int src)
{
    return in + (long long)src * kRowAlign;
}

// Programmatic dependent launch of consecutive steps.  A step kernel lets
// the next step's grid be scheduled once all of its own blocks have started
// (so the next step's blocks fill the SMs its last wave leaves idle and
// load their row records), and every step waits for the previous kernel to
// complete, its memory visible, before it reads or writes anything that
// kernel reads or writes.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ T lagged(const T *U1, const T *U2, int idx)
{
    return T(0.5) * (U1[idx] + U2[idx]);
}

// Pull-stream the Q populations of one species at (row, x): direction i
// comes from column x, x - 1 or x + 1 of the source row R.src[i] of `in`, decoded against
// the source references `dec` for reduced-precision storage.
template <int Q, typename T, typename S>
__device__ __forceinline__ void pull(const S *__restrict__ in, const RowInfo &R, int x, int xm1,
                                     int xp1, const float *dec, float inv_scale, T g[Q])
{
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int xs = ((R.xm >> i) & 1u) ? xm1 : (((R.xp >> i) & 1u) ? xp1 : x);
        if constexpr (Storage<S>::kRef)
            g[i] = Storage<S>::load(src_row(in, R.src[i]) + xs) * inv_scale + __ldg(dec + i);
        else
            g[i] = Storage<S>::load(src_row(in, R.src[i]) + xs);
    }
}

// Water cell given its streamed populations g: moments, interface friction,
// Guo velocity.  U1/U2 are the velocities of the two steps before the time
// level of g; R is the row's table.
template <int Q, typename T>
__device__ __forceinline__ void water_math(const StepArgs<T> &p, const T *Uw1, const T *Uw2,
                                           const T *Us1, const T *Us2, const RowInfo &R, int x,
                                           const T g[Q], Cell<T> &c, T j[3])
{
    moments<Q, T>(g, c.drho, j);
    c.F[0] = p.G[0];
    c.F[1] = p.G[1];
    c.F[2] = p.G[2];
    const int slot = R.slot;
    if (slot >= 0) {
        const int ns_w = p.n_slots[kFluid], ns_s = p.n_slots[kSolid], nxp = p.nxp;
        const int nface = R.nface;
        for (int a = 0; a < 3; ++a) {
            const T uw = lagged(Uw1, Uw2, (a * ns_w + slot) * nxp + x);
            T f = T(0);
            for (int k = 0; k < nface; ++k) {
                const int q = R.partner[k];
                const T de = uw - lagged(Us1, Us2, (a * ns_s + q) * nxp + x);
                const T dp = uw - lagged(Us1, Us2, ((a + 3) * ns_s + q) * nxp + x);
                f -= p.g_we * de + p.g_wp * dp;
            }
            c.F[a] += f;
        }
    }
    const T rinv = T(1) / (p.rho0 + c.drho);
#pragma unroll
    for (int a = 0; a < 3; ++a) c.u[a] = (j[a] + T(0.5) * c.F[a]) * rinv;
}

// Electrons and phonons of one solid cell given their streamed populations.
template <int Q, typename T>
__device__ __forceinline__ void solid_math(const StepArgs<T> &p, const T *Uw1, const T *Uw2,
                                           const T *Us1, const T *Us2, const RowInfo &R, int x,
                                           const T ge[Q], const T gp[Q], Cell<T> &ce,
                                           Cell<T> &cp, T je[3], T jp[3])
{
    moments<Q, T>(ge, ce.drho, je);
    moments<Q, T>(gp, cp.drho, jp);
    T Fe[3] = {T(0), T(0), T(0)}, Fp[3] = {T(0), T(0), T(0)};
    const int slot = R.slot;
    if (slot >= 0) {
        const int ns_w = p.n_slots[kFluid], ns_s = p.n_slots[kSolid], nxp = p.nxp;
        const int nface = R.nface;
        for (int a = 0; a < 3; ++a) {
            const T ue = lagged(Us1, Us2, (a * ns_s + slot) * nxp + x);
            const T up = lagged(Us1, Us2, ((a + 3) * ns_s + slot) * nxp + x);
            T fe = T(0), fp = T(0);
            for (int k = 0; k < nface; ++k) {
                const T uw = lagged(Uw1, Uw2, (a * ns_w + R.partner[k]) * nxp + x);
                fe += p.g_we * (uw - ue);
                fp += p.g_wp * (uw - up);
            }
            Fe[a] = fe;
            Fp[a] = fp;
        }
    }
    // Trapezoidal e-p friction and sinks, solved exactly per component:
    // (a + k + se) ue - k up = Je,  -k ue + (b + k + sp) up = Jp.
    const T ra = p.rho0 + ce.drho, rb = p.rho0 + cp.drho;
    const T k = T(0.5) * p.g_ep, se = T(0.5) * p.g_ec, sp = T(0.5) * p.g_pc;
    const T A = ra + k + se, B = rb + k + sp;
    const T Dinv = T(1) / (A * B - k * k);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T Je = je[a] + T(0.5) * Fe[a];
        const T Jp = jp[a] + T(0.5) * Fp[a];
        const T ue = (B * Je + k * Jp) * Dinv;
        const T up = (A * Jp + k * Je) * Dinv;
        ce.u[a] = ue;
        cp.u[a] = up;
        ce.F[a] = Fe[a] - p.g_ep * (ue - up) - p.g_ec * ue;
        cp.F[a] = Fp[a] + p.g_ep * (ue - up) - p.g_pc * up;
    }
}

// ---------------------------------------------------------------------------
// Debug builds (-DKLB_BOUNDS=1; the sanitiser is not available) check, before
// a thread touches anything, that every index it will derive from its row
// record lies inside its array: the row, the Q source offsets (whole rows of
// the population array), the x positions (inside the padded row), the
// interface slot and the partner slots.  A failure records its site in the
// lattice's error word (klb_bounds_status) and the thread continues on row 0
// as a dead thread, touching only valid memory.  Normal builds compile
// nothing of this.
enum BoundsSite { kBadRow = 1, kBadSource = 2, kBadX = 3, kBadSlot = 4, kBadPartner = 5, kBadFaces = 6 };

template <int Q, typename T>
__device__ __noinline__ bool row_indices_ok(const StepArgs<T> &p, bool water, int row, int xmin, int xmax)
{
    const int cls = water ? kFluid : kSolid, other = 1 - cls;
    unsigned site = 0;
    if (row < 0 || row >= p.n_rows[cls]) {
        site = kBadRow;
    } else if (xmin < 0 || xmax >= p.nxp) {
        site = kBadX;
    } else {
        const RowInfo &R = p.rows[cls][row];
        const int unit = p.nxp / kRowAlign;
        const long long hi = ((long long)Q * p.n_rows[cls] - 1) * unit;
        for (int i = 0; i < Q && !site; ++i) {
            const int v = R.src[i];
            if (v < 0 || v > hi || v % unit) site = kBadSource;
        }
        if (!site && R.slot >= p.n_slots[cls]) site = kBadSlot;
        if (!site && (R.nface < 0 || R.nface > kMaxFaces)) site = kBadFaces;
        for (int k = 0; !site && k < R.nface; ++k)
            if (R.slot >= 0 && (R.partner[k] < 0 || R.partner[k] >= p.n_slots[other])) site = kBadPartner;
    }
    if (site) atomicCAS(p.bounds_err, 0u, site);
    return site == 0;
}

// ---------------------------------------------------------------------------
// Block reductions (fixed order).

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block sums of the observation pass (one row chunk per block, so the row
// class and flags are block-uniform; ncell = the thread's live cells).  Only the sums that can be non-zero
// for the block's class run a warp reduction (FP64 throughput on GB300 is a
// small fraction of FP32); the slip-fit count and distance moments and the wall-row count
// follow from the number of live cells and the row's d^2, the fit and
// wall-row u_x sums are the u_x sum itself (every cell of such a row adds
// its u_x to both), and non-finite values are counted with block-wide
// predicate counts.  Each entry equals what a reduction of the per-cell
// values gives.
__device__ inline void observe_reduce_store(const double (&s)[kNumSums], bool water, int flags, double d2,
                                            int ncell, double *out)
{
    __shared__ double red[kNumSums][kBlockX / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    const bool fit = water && (flags & kFitRow), wall = water && (flags & kWallRow);
    const uint32_t sel =
        water ? (1u << kSumUxFluid) | (1u << kSumMomW) | (1u << kSumMassW) | (1u << kSumResidual) |
                    (fit ? (1u << kSumFitUD2) : 0u)
              : (1u << kSumUxE) | (1u << kSumUxP) | (1u << kSumMomE) | (1u << kSumMomP) | (1u << kSumMassE) |
                    (1u << kSumMassP) | (1u << kSumResidual);
    const int cnt = __syncthreads_count(ncell >= 1) + __syncthreads_count(ncell >= 2);  // live cells
    // per-thread counts of up to four species-cells (two cells of two species)
    auto count4 = [](double v) {
        return __syncthreads_count(v >= 1.0) + __syncthreads_count(v >= 2.0) + __syncthreads_count(v >= 3.0) +
               __syncthreads_count(v >= 4.0);
    };
    const int nonfinite = count4(s[kSumNonfinite]);
    const int clipped = count4(s[kSumClipped]);
#pragma unroll
    for (int k = 0; k < kNumSums; ++k) {
        if (!((sel >> k) & 1u)) continue;
        const double v = (k == kSumResidual) ? warp_max(s[k]) : warp_sum(s[k]);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kNumSums) {
        const int k = threadIdx.x;
        auto total = [&](int kk) {
            double v = red[kk][0];
            for (int w = 1; w < nwarps; ++w) v = (kk == kSumResidual) ? fmax(v, red[kk][w]) : v + red[kk][w];
            return v;
        };
        double v = 0.0;
        if ((sel >> k) & 1u)
            v = total(k);
        else if (k == kSumFitN)
            v = fit ? (double)cnt : 0.0;
        else if (k == kSumFitD2)
            v = fit ? cnt * d2 : 0.0;
        else if (k == kSumFitD4)
            v = fit ? cnt * (d2 * d2) : 0.0;
        else if (k == kSumFitU)
            v = fit ? total(kSumUxFluid) : 0.0;
        else if (k == kSumWallN)
            v = wall ? (double)cnt : 0.0;
        else if (k == kSumWallU)
            v = wall ? total(kSumUxFluid) : 0.0;
        else if (k == kSumNonfinite)
            v = (double)nonfinite;
        else if (k == kSumClipped)
            v = (double)clipped;
        out[k] = v;
    }
}

// x-sums over one warp (a 32-wide x segment of a row) of NV values per
// thread, written by lane 0 to out[0 .. NV): the partial sums that reference
// refreshes reduce.  Lanes past the end of the row contribute zeros.
template <int NV>
__device__ __forceinline__ void warp_xsum(const float (&v)[NV], float *out)
{
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const float s = warp_sumf(v[k]);
        if ((threadIdx.x & 31) == 0) out[k] = s;
    }
}

// Segment (32-wide x run of a row) of the calling warp, or -1 when the warp
// lies past the end of its row.
template <typename T>
__device__ __forceinline__ int warp_segment(const StepArgs<T> &p, bool water, int row, int x_lane0)
{
    const int xw = x_lane0 - (threadIdx.x & 31);
    if (xw >= p.nx) return -1;
    return (water ? 0 : p.nseg_w) + row * p.nch32 + xw / 32;
}

template <typename T>
__device__ __forceinline__ bool finite3(const Cell<T> &c)
{
    return isfinite((double)c.drho) && isfinite((double)c.u[0]) && isfinite((double)c.u[1]) &&
           isfinite((double)c.u[2]);
}

// ---------------------------------------------------------------------------
// Observation and field passes.

template <int Q, typename T, typename S, int MODE>
__global__ void __launch_bounds__(kBlockX, (sizeof(T) == 4 ? 8 : 1)) k_lattice(const StepArgs<T> p)
{
    const int b = blockIdx.x;
    const bool water = b < p.nbw;
    const int bb = water ? b : b - p.nbw;
    int row = bb / p.nchunk;
    const int x = (bb - row * p.nchunk) * blockDim.x + threadIdx.x;
    bool live = x < p.nx;
    if constexpr (KLB_BOUNDS) {
        if (live && !row_indices_ok<Q>(p, water, row, 0, x)) {
            live = false;
            row = 0;
        }
    }
    const float inv = p.inv_scale;

    double s[kNumSums];
    if (MODE == kModeObserve) {
#pragma unroll
        for (int k = 0; k < kNumSums; ++k) s[k] = 0.0;
    }

    if (live) {
        const int xm1 = x == 0 ? p.nx - 1 : x - 1;
        const int xp1 = x == p.nx - 1 ? 0 : x + 1;
        const int nxp = p.nxp;
        if (water) {
            const RowInfo &R = p.rows[kFluid][row];
            T g[Q], j[3];
            Cell<T> c;
            pull<Q, T, S>(static_cast<const S *>(p.in[0]), R, x, xm1, xp1,
                          ref_row<T, S>(p.dec_in[0], row), inv, g);
            water_math<Q, T>(p, p.U1[kFluid], p.U2[kFluid], p.U1[kSolid], p.U2[kSolid], R, x, g, c, j);
            if (MODE == kModeField) {
                T *f = p.field;
                f[row * nxp + x] = c.drho;
                for (int a = 0; a < 3; ++a) f[((size_t)(a + 1) * p.n_rows[kFluid] + row) * nxp + x] = c.u[a];
            } else {
                const double ux = (double)c.u[0];
                const double rho = (double)(p.rho0 + c.drho);
                s[kSumUxFluid] = ux;
                s[kSumMomW] = rho * ux;
                s[kSumMassW] = (double)c.drho;
                s[kSumNonfinite] = finite3(c) ? 0.0 : 1.0;
                s[kSumClipped] = clipped_cell<Q, S>(static_cast<const S *>(p.in[0]), R, x, xm1, xp1) ? 1.0 : 0.0;
                if (R.flags & kFitRow) {
                    const double d2 = (double)R.d2;
                    s[kSumFitN] = 1.0;
                    s[kSumFitD2] = d2;
                    s[kSumFitD4] = d2 * d2;
                    s[kSumFitU] = ux;
                    s[kSumFitUD2] = ux * d2;
                }
                if (R.flags & kWallRow) {
                    s[kSumWallN] = 1.0;
                    s[kSumWallU] = ux;
                }
                if (p.residual_valid) {
                    Cell<T> cprev;
                    pull<Q, T, S>(static_cast<const S *>(p.in_prev[0]), R, x, xm1, xp1,
                                  ref_row<T, S>(p.dec_prev[0], row), inv, g);
                    water_math<Q, T>(p, p.U2[kFluid], p.U3[kFluid], p.U2[kSolid], p.U3[kSolid], R, x,
                                     g, cprev, j);
                    s[kSumResidual] = fabs(ux - (double)cprev.u[0]);
                }
            }
        } else {
            const RowInfo &R = p.rows[kSolid][row];
            T ge[Q], gp[Q], je[3], jp[3];
            Cell<T> ce, cp;
            pull<Q, T, S>(static_cast<const S *>(p.in[1]), R, x, xm1, xp1,
                          ref_row<T, S>(p.dec_in[1], row), inv, ge);
            pull<Q, T, S>(static_cast<const S *>(p.in[2]), R, x, xm1, xp1,
                          ref_row<T, S>(p.dec_in[2], row), inv, gp);
            solid_math<Q, T>(p, p.U1[kFluid], p.U2[kFluid], p.U1[kSolid], p.U2[kSolid], R, x, ge,
                             gp, ce, cp, je, jp);
            if (MODE == kModeField) {
                const int nrw = p.n_rows[kFluid], nrs = p.n_rows[kSolid];
                T *fe = p.field + (size_t)4 * nrw * nxp;
                T *fp = fe + (size_t)4 * nrs * nxp;
                fe[row * nxp + x] = ce.drho;
                fp[row * nxp + x] = cp.drho;
                for (int a = 0; a < 3; ++a) {
                    fe[((size_t)(a + 1) * nrs + row) * nxp + x] = ce.u[a];
                    fp[((size_t)(a + 1) * nrs + row) * nxp + x] = cp.u[a];
                }
            } else {
                const double ue = (double)ce.u[0], up = (double)cp.u[0];
                s[kSumUxE] = ue;
                s[kSumUxP] = up;
                s[kSumMomE] = (double)(p.rho0 + ce.drho) * ue;
                s[kSumMomP] = (double)(p.rho0 + cp.drho) * up;
                s[kSumMassE] = (double)ce.drho;
                s[kSumMassP] = (double)cp.drho;
                s[kSumNonfinite] = (finite3(ce) ? 0.0 : 1.0) + (finite3(cp) ? 0.0 : 1.0);
                s[kSumClipped] = (clipped_cell<Q, S>(static_cast<const S *>(p.in[1]), R, x, xm1, xp1) ? 1.0 : 0.0) +
                                 (clipped_cell<Q, S>(static_cast<const S *>(p.in[2]), R, x, xm1, xp1) ? 1.0 : 0.0);
                if (p.residual_valid) {
                    Cell<T> pe, pp;
                    pull<Q, T, S>(static_cast<const S *>(p.in_prev[1]), R, x, xm1, xp1,
                                  ref_row<T, S>(p.dec_prev[1], row), inv, ge);
                    pull<Q, T, S>(static_cast<const S *>(p.in_prev[2]), R, x, xm1, xp1,
                                  ref_row<T, S>(p.dec_prev[2], row), inv, gp);
                    solid_math<Q, T>(p, p.U2[kFluid], p.U3[kFluid], p.U2[kSolid], p.U3[kSolid], R, x,
                                     ge, gp, pe, pp, je, jp);
                    s[kSumResidual] = fmax(fabs(ue - (double)pe.u[0]), fabs(up - (double)pp.u[0]));
                }
            }
        }
    }
    if (MODE == kModeObserve) {
        const RowInfo &Rb = p.rows[water ? kFluid : kSolid][row];
        observe_reduce_store(s, water, water ? Rb.flags : 0, (double)Rb.d2, live ? 1 : 0,
                             p.partials + (size_t)b * kNumSums);
    }
}

// Start from the local equilibrium of the fields (drho, u) staged in p.field
// (the layout the field pass writes): the state buffer p.out and the
// lagged-velocity slot p.U0 are filled.  With ACC, nothing is stored and the
// per-block x-sums of the equilibria go to p.acc instead (the first half of a
// reduced-precision start, which needs the references before encoding).
template <int Q, typename T, typename S, bool ACC>
__global__ void __launch_bounds__(kBlockX) k_init(const StepArgs<T> p)
{
    const int b = blockIdx.x;
    const bool water = b < p.nbw;
    const int bb = water ? b : b - p.nbw;
    int row = bb / p.nchunk;
    const int x = (bb - row * p.nchunk) * blockDim.x + threadIdx.x;
    bool live = x < p.nx;
    if constexpr (KLB_BOUNDS) {
        if (live && !row_indices_ok<Q>(p, water, row, x, x)) {
            live = false;
            row = 0;
        }
    }
    const int nxp = p.nxp;
    const int nrw = p.n_rows[kFluid], nrs = p.n_rows[kSolid];
    const int cls = water ? kFluid : kSolid;
    const RowInfo &R = p.rows[cls][row];
    float sums[2 * Q];
#pragma unroll
    for (int k = 0; k < 2 * Q; ++k) sums[k] = 0.f;
    const int nsp = water ? 1 : 2;
    for (int k = 0; k < nsp; ++k) {
        const int s = water ? 0 : 1 + k;
        const int nr = water ? nrw : nrs;
        const T *f = p.field;
        if (s >= 1) f += (size_t)4 * nrw * nxp;
        if (s == 2) f += (size_t)4 * nrs * nxp;
        if (!live) continue;
        Cell<T> c;
        c.drho = f[row * nxp + x];
        for (int a = 0; a < 3; ++a) {
            c.u[a] = f[((size_t)(a + 1) * nr + row) * nxp + x];
            c.F[a] = T(0);
        }
        // om = 1 and F = 0 make the collision produce exactly g^eq, whose
        // moments are drho and rho u.
        T g[Q], jeq[3];
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = T(0);
        for (int a = 0; a < 3; ++a) jeq[a] = (p.rho0 + c.drho) * c.u[a];
        collide<Q, T>(g, c, jeq, p.rho0, T(1), s == 2 ? p.q_p : T(1));
        if constexpr (ACC) {
#pragma unroll
            for (int i = 0; i < Q; ++i) sums[k * Q + i] = float(g[i]);
        } else {
            store_cell<Q, T, S>(g, static_cast<S *>(p.out[s]), nr * nxp, row * nxp + x,
                                ref_row<T, S>(p.enc_out[s], row), p.scale);
            if (R.slot >= 0) {
                const int ns = p.n_slots[cls];
                const int off = water ? 0 : 3 * k;
                for (int a = 0; a < 3; ++a) p.U0[cls][((a + off) * ns + R.slot) * nxp + x] = c.u[a];
            }
        }
    }
    if constexpr (ACC) {
        const int seg = warp_segment(p, water, row, x);
        if (seg >= 0) warp_xsum<2 * Q>(sums, p.acc + (size_t)seg * 2 * Q);
    }
}

// ---------------------------------------------------------------------------
// Step kernel.
//
// One block per work item (one row, up to 128 threads along x).  With FP32
// arithmetic a thread updates two adjacent cells (klb_step_pair.cuh), in
// FP64 one (step_body below).  Memory parallelism comes from residency: the
// FP32-arithmetic kernel is held to 96 registers (5 blocks of 128 threads
// per SM; a few spilled values cost less than the occupancy they buy), and
// every thread issues its loads back to back.  The row table is read with
// 16-byte loads (one 128-byte line per row, cached); the x shift of each
// direction is a compile-time constant except on the few rows where an
// x-moving population bounces back.  A solid cell streams, and takes the
// moments of, both its electrons and phonons, then collides and stores the
// electrons before pulling the phonons a second time (the lines are still
// cached), so that at most Q populations are live at once.  With ACC the
// block also writes the x-sums of its post-collision populations to p.acc
// for the next reference refresh of reduced-precision storage.

template <int Q, typename T, typename S>
__device__ __forceinline__ T pull_one(const S *__restrict__ in, int src, int xs, const float *dec,
                                      int i, float inv_scale)
{
    if constexpr (Storage<S>::kRef)
        return Storage<S>::load(src_row(in, src) + xs) * inv_scale + __ldg(dec + i);
    else
        return Storage<S>::load(src_row(in, src) + xs);
}

template <int Q, typename T, typename S>
__device__ __forceinline__ void pull_row(const S *__restrict__ in, const int src[Q], uint32_t xm,
                                         uint32_t xp, bool xbounce, int x, int pm, int pp,
                                         const float *dec, float inv_scale, T g[Q])
{
    if (!xbounce) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int xs = cx<Q>(i) > 0 ? pm : (cx<Q>(i) < 0 ? pp : x);
            g[i] = pull_one<Q, T, S>(in, src[i], xs, dec, i, inv_scale);
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int xs = ((xm >> i) & 1u) ? pm : (((xp >> i) & 1u) ? pp : x);
            g[i] = pull_one<Q, T, S>(in, src[i], xs, dec, i, inv_scale);
        }
    }
}

// The kernel reads the row record as eight 16-byte words.
static_assert(offsetof(RowInfo, xm) == 19 * 4 && offsetof(RowInfo, xp) == 20 * 4 &&
                  offsetof(RowInfo, slot) == 21 * 4 && offsetof(RowInfo, flags) == 28 * 4 &&
                  offsetof(RowInfo, cs) == 29 * 4,
              "row record layout");

// ---------------------------------------------------------------------------
// Thermal fluctuations of the water (Eq. 6, Eq. 17), read as the standard
// fluctuating lattice Boltzmann method: after the collision every
// non-conserved moment of the water populations gets the Gaussian noise its
// relaxation removes, i.e. g*_i += A (a_i - w_i sum_j a_j - 3 w_i c_i . sum_j
// c_j a_j) with a_i = sqrt(w_i) z_i, z_i independent standard normals and
// A = sqrt(3 rho0 kT omega (2 - omega)).  The normals of cell (x, cs) at step
// n come from the Philox-4x32-10 counter-based generator (Salmon et al.,
// SC 2011: ten rounds of two 32x32->64-bit products recombined as
// (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), the key bumped by the Weyl
// constants between rounds) with counter (x + nx cs, n mod 2^32, n / 2^32,
// block) and the seed as key; each word r gives u = (r + 1/2) 2^-32 and
// pairs of uniforms give two normals by Box-Muller.

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Two normals from two generator words (Box-Muller).  FP32: u = r 2^-32 +
// 2^-33 (exact for small r, where the logarithm is sensitive); the hardware
// logarithm and sine/cosine (relative error near 1e-6, far below what the
// statistics of the noise can resolve), the angle taken as
// 2 pi (u2 - 1/2) in [-pi, pi), where the fast sine/cosine are accurate,
// and the half turn undone by negating both.
__device__ __forceinline__ void box_muller(uint32_t r1, uint32_t r2, float &z1, float &z2)
{
    const float u1 = fmaf(__uint2float_rn(r1), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
    const float u2 = fmaf(__uint2float_rn(r2), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
    const float R = sqrtf(-2.f * __logf(u1));
    float sn, cs;
    __sincosf(6.2831853071795865f * (u2 - 0.5f), &sn, &cs);
    z1 = -R * cs;
    z2 = -R * sn;
}
__device__ __forceinline__ void box_muller(uint32_t r1, uint32_t r2, double &z1, double &z2)
{
    const double u1 = ((double)r1 + 0.5) * 2.3283064365386963e-10;
    const double u2 = ((double)r2 + 0.5) * 2.3283064365386963e-10;
    const double R = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    z1 = R * cs;
    z2 = R * sn;
}

// sqrt(w_i) (textbook weights 1/3, 1/18, 1/36 and 4/9, 1/9, 1/36).
template <int Q>
__host__ __device__ constexpr double sqrt_wt(int i)
{
    return Q == 19 ? (i == 0 ? 0.57735026918962576451 : (i <= 6 ? 0.23570226039551584147 : 1.0 / 6.0))
                   : (i == 0 ? 2.0 / 3.0 : (i <= 4 ? 1.0 / 3.0 : 1.0 / 6.0));
}

// Calls f(i, a_i) for the Q weighted normals a_i = sqrt(w_i) z_i of a cell.
template <int Q, typename T, typename F>
__device__ __forceinline__ void weighted_normals(uint32_t cell, uint32_t slo, uint32_t shi, uint32_t k0,
                                                 uint32_t k1, F f)
{
#pragma unroll
    for (int b = 0; b < (Q + 3) / 4; ++b) {
        const uint4 r = philox4x32_10(make_uint4(cell, slo, shi, (uint32_t)b), k0, k1);
        T z[4];
        box_muller(r.x, r.y, z[0], z[1]);
        box_muller(r.z, r.w, z[2], z[3]);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int i = 4 * b + h;
            if (i < Q) f(i, T(sqrt_wt<Q>(i)) * z[h]);
        }
    }
}

// Calls add(i, xi_i) with the noise of one water cell (see above); the
// normals are drawn once and held for the projection.
template <int Q, typename T, typename F>
__device__ __forceinline__ void thermal_noise(const StepArgs<T> &p, uint32_t cell, F add)
{
    T S0 = T(0), S1[3] = {T(0), T(0), T(0)}, a[Q];
    weighted_normals<Q, T>(cell, p.step_lo, p.step_hi, p.key[0], p.key[1], [&](int i, T v) {
        a[i] = v;
        S0 += v;
        if (cx<Q>(i)) S1[0] += T(cx<Q>(i)) * v;
        if (cy<Q>(i)) S1[1] += T(cy<Q>(i)) * v;
        if (cz<Q>(i)) S1[2] += T(cz<Q>(i)) * v;
    });
    const T A = p.noise_amp;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T w = T(wt<Q>(i));
        const T cS = T(cx<Q>(i)) * S1[0] + T(cy<Q>(i)) * S1[1] + T(cz<Q>(i)) * S1[2];
        add(i, A * (a[i] - w * S0 - T(3) * w * cS));
    }
}

template <typename T, typename S>
constexpr int step_min_blocks()
{
    return sizeof(T) == 8 ? 4 : 5;
}

template <int Q, typename T, typename S, bool ACC, bool NOISE = false>
__device__ __forceinline__ void step_body(const StepArgs<T> &p, int b)
{
    // solid blocks (two species each, the heavier work) first, so that the
    // grid's last wave holds the lighter water blocks
    const int nsb = p.n_rows[kSolid] * p.snchunk_s;
    const bool water = b >= nsb;
    const int bb = water ? b - nsb : b;
    const int nch = water ? p.snchunk_w : p.snchunk_s;
    int row = bb / nch;
    int x = (bb - row * nch) * blockDim.x + threadIdx.x;
    const int x_lane = x;
    bool live = x < p.nx;
    if constexpr (KLB_BOUNDS) {
        if (live && !row_indices_ok<Q>(p, water, row, 0, x)) {
            live = false;
            row = 0;
        }
    }
    if constexpr (!ACC) {
        if (!live) return;  // no warp-wide operation follows
    } else {
        if (!live) x = 0;   // computes nothing, but joins the warp reduction
    }
    const int pm = x == 0 ? p.nx - 1 : x - 1;
    const int pp = x == p.nx - 1 ? 0 : x + 1;
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
    const uint32_t xm = (uint32_t)src[19];  // the 20th word of a row is its xm mask
    const int4 q5 = __ldg(t4 + 5);          // xp, slot, nface, partner[0]
    const int4 q7 = __ldg(t4 + 7);          // flags, cs, pad, pad
    const uint32_t xp = (uint32_t)q5.x;
    const bool xbounce = (q7.x & kXBounce) != 0;
    pdl_wait();  // populations, lagged velocities and references below

    if (water) {
        T g[Q], j[3];
        Cell<T> c;
        if (!ACC || live) {
            pull_row<Q, T, S>(static_cast<const S *>(p.in[0]), src, xm, xp, xbounce, x, pm, pp,
                              ref_row<T, S>(p.dec_in[0], row), inv, g);
            water_math<Q, T>(p, p.U1[kFluid], p.U2[kFluid], p.U1[kSolid], p.U2[kSolid], R, x, g, c, j);
            if (q5.y >= 0) {
                const int ns = p.n_slots[kFluid];
                for (int a = 0; a < 3; ++a) p.U0[kFluid][(a * ns + q5.y) * nxp + x] = c.u[a];
            }
            collide<Q, T>(g, c, j, p.rho0, p.om[0]);
            if constexpr (NOISE)
                thermal_noise<Q, T>(p, (uint32_t)x + (uint32_t)p.nx * (uint32_t)q7.y,
                                    [&](int i, T v) { g[i] += v; });
            store_cell<Q, T, S>(g, static_cast<S *>(p.out[0]), p.n_rows[kFluid] * nxp,
                                row * nxp + x, ref_row<T, S>(p.enc_out[0], row), sc);
        }
        if constexpr (ACC) {
            float acc[2 * Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                acc[i] = live ? float(g[i]) : 0.f;
                acc[Q + i] = 0.f;
            }
            const int seg = warp_segment(p, true, row, x_lane);
            if (seg >= 0) warp_xsum<2 * Q>(acc, p.acc + (size_t)seg * 2 * Q);
        }
        return;
    }

    T ge[Q], gp[Q], je[3], jp[3];
    Cell<T> ce, cp;
    float acc[ACC ? 2 * Q : 1];
    if (!ACC || live) {
        pull_row<Q, T, S>(static_cast<const S *>(p.in[1]), src, xm, xp, xbounce, x, pm, pp,
                          ref_row<T, S>(p.dec_in[1], row), inv, ge);
        pull_row<Q, T, S>(static_cast<const S *>(p.in[2]), src, xm, xp, xbounce, x, pm, pp,
                          ref_row<T, S>(p.dec_in[2], row), inv, gp);
        solid_math<Q, T>(p, p.U1[kFluid], p.U2[kFluid], p.U1[kSolid], p.U2[kSolid], R, x, ge, gp,
                         ce, cp, je, jp);
        if (q5.y >= 0) {
            const int ns = p.n_slots[kSolid];
            for (int a = 0; a < 3; ++a) {
                p.U0[kSolid][(a * ns + q5.y) * nxp + x] = ce.u[a];
                p.U0[kSolid][((a + 3) * ns + q5.y) * nxp + x] = cp.u[a];
            }
        }
        const int stride = p.n_rows[kSolid] * nxp, base = row * nxp + x;
        collide<Q, T>(ge, ce, je, p.rho0, p.om[1]);
        store_cell<Q, T, S>(ge, static_cast<S *>(p.out[1]), stride, base,
                            ref_row<T, S>(p.enc_out[1], row), sc);
        if constexpr (ACC) {
#pragma unroll
            for (int i = 0; i < Q; ++i) acc[i] = float(ge[i]);
        }
        pull_row<Q, T, S>(static_cast<const S *>(p.in[2]), src, xm, xp, xbounce, x, pm, pp,
                          ref_row<T, S>(p.dec_in[2], row), inv, gp);
        collide<Q, T>(gp, cp, jp, p.rho0, p.om[2], p.q_p);
        store_cell<Q, T, S>(gp, static_cast<S *>(p.out[2]), stride, base,
                            ref_row<T, S>(p.enc_out[2], row), sc);
        if constexpr (ACC) {
#pragma unroll
            for (int i = 0; i < Q; ++i) acc[Q + i] = float(gp[i]);
        }
    } else if constexpr (ACC) {
#pragma unroll
        for (int k = 0; k < 2 * Q; ++k) acc[k] = 0.f;
    }
    if constexpr (ACC) {
        const int seg = warp_segment(p, false, row, x_lane);
        if (seg >= 0) warp_xsum<2 * Q>(acc, p.acc + (size_t)seg * 2 * Q);
    }
}

}  // namespace klb

#include "klb_step_pair.cuh"

namespace klb {

// FP32 arithmetic: two cells per thread (klb_step_pair.cuh); FP64: one.
template <int Q, typename T, typename S, bool ACC, bool NOISE = false>
__device__ __forceinline__ void step_cells_body(const StepArgs<T> &p, int b)
{
    if constexpr (sizeof(T) == 4)
        step_body2<Q, S, ACC, NOISE>(p, b);
    else
        step_body<Q, T, S, ACC, NOISE>(p, b);
}

template <int Q, typename T, typename S, bool ACC, bool NOISE = false>
__global__ void __launch_bounds__(kBlockX, (step_min_blocks<T, S>())) k_step(const StepArgs<T> p)
{
    pdl_launch_dependents();
    step_cells_body<Q, T, S, ACC, NOISE>(p, blockIdx.x);
}

// Launch of a step kernel that may begin while the previous kernel of the
// stream finishes (see pdl_wait); batched steps are launched the same way.
template <typename A>
cudaError_t launch_step(void (*kernel)(A), int nblocks, int bx, cudaStream_t s, const A &a)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nblocks);
    cfg.blockDim = dim3((unsigned)bx);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

// Many lattices in one launch: the block finds its lattice as the number of
// lattices after the first whose first block is at or before its own
// (prefix[] is increasing), counted by all threads at once — one round of
// independent loads instead of a chain of dependent ones — and works from a
// shared-memory copy of that lattice's arguments.
template <int Q, typename T, typename S, bool ACC>
__global__ void __launch_bounds__(kBlockX, (step_min_blocks<T, S>()))
    k_step_batch(const StepArgs<T> *__restrict__ table, const int *__restrict__ prefix, int n)
{
    pdl_launch_dependents();
    __shared__ StepArgs<T> sp;
    __shared__ int s_lid;
    if (threadIdx.x == 0) s_lid = 0;
    __syncthreads();
    int c = 0;
    for (int m = 1 + (int)threadIdx.x; m < n; m += blockDim.x) c += __ldg(prefix + m) <= (int)blockIdx.x;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s_lid, c);
    __syncthreads();
    const int lid = s_lid;
    static_assert(sizeof(StepArgs<T>) % 16 == 0, "argument record in 16-byte words");
    const int4 *src = reinterpret_cast<const int4 *>(table + lid);
    int4 *dst = reinterpret_cast<int4 *>(&sp);
    for (int k = threadIdx.x; k < (int)(sizeof(StepArgs<T>) / 16); k += blockDim.x) dst[k] = __ldg(src + k);
    __syncthreads();
    step_cells_body<Q, T, S, ACC>(sp, (int)blockIdx.x - __ldg(prefix + lid));
}

// ---------------------------------------------------------------------------
// Reference refresh of reduced-precision storage.  A row's new reference for
// direction i is the x-average of its post-collision populations, summed in
// fixed order from the per-block x-sums; the decode table holds, for every
// (row, direction), the reference of the population it pulls.

template <int Q, typename T>
__global__ void k_ref_sum(const StepArgs<T> p, float *enc0, float *enc1, float *enc2)
{
    const int nrw = p.n_rows[kFluid], nrs = p.n_rows[kSolid];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = (nrw + 2 * nrs) * Q;
    if (k >= total) return;
    const int r = k / Q, i = k - r * Q;
    int s, row;
    if (r < nrw) {
        s = 0;
        row = r;
    } else if (r < nrw + nrs) {
        s = 1;
        row = r - nrw;
    } else {
        s = 2;
        row = r - nrw - nrs;
    }
    const int seg0 = (s == 0 ? 0 : p.nseg_w) + row * p.nch32;
    const int off = s == 2 ? Q + i : i;
    float sum = 0.f;
    for (int c = 0; c < p.nch32; ++c) sum += p.acc[(size_t)(seg0 + c) * 2 * Q + off];
    float *enc = s == 0 ? enc0 : (s == 1 ? enc1 : enc2);
    enc[(size_t)row * kRefStride + i] = sum / (float)p.nx;
}

template <int Q, typename T>
__global__ void k_ref_dec(const StepArgs<T> p, const float *enc0, const float *enc1,
                          const float *enc2, float *dec0, float *dec1, float *dec2)
{
    const int nrw = p.n_rows[kFluid], nrs = p.n_rows[kSolid];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = (nrw + 2 * nrs) * Q;
    if (k >= total) return;
    const int r = k / Q, i = k - r * Q;
    const int s = r < nrw ? 0 : (r < nrw + nrs ? 1 : 2);
    const int row = s == 0 ? r : (s == 1 ? r - nrw : r - nrw - nrs);
    const int cls = s == 0 ? kFluid : kSolid;
    const int nr = s == 0 ? nrw : nrs;
    const int q = p.rows[cls][row].src[i] / (p.nxp / kRowAlign);  // sdir * nr + srow
    const int sdir = q / nr, srow = q - sdir * nr;
    const float *enc = s == 0 ? enc0 : (s == 1 ? enc1 : enc2);
    float *dec = s == 0 ? dec0 : (s == 1 ? dec1 : dec2);
    dec[(size_t)row * kRefStride + i] = enc[(size_t)srow * kRefStride + sdir];
}

// ---------------------------------------------------------------------------
// Launch templates (instantiated per lattice).

template <int Q, typename T, typename S>
cudaError_t launch_q(const void *args, int mode, int nblocks, int bx, cudaStream_t s)
{
    const StepArgs<T> &a = *static_cast<const StepArgs<T> *>(args);
    switch (mode) {
    case kModeStep:
        return launch_step<StepArgs<T>>(k_step<Q, T, S, false>, nblocks, bx, s, a);
    case kModeStepAcc:
        if constexpr (Storage<S>::kRef)
            return launch_step<StepArgs<T>>(k_step<Q, T, S, true>, nblocks, bx, s, a);
        else
            return cudaErrorInvalidValue;
    case kModeStepNoise:
        if constexpr (!Storage<S>::kRef)
            return launch_step<StepArgs<T>>(k_step<Q, T, S, false, true>, nblocks, bx, s, a);
        else
            return cudaErrorInvalidValue;
    case kModeObserve:
        // FP32 arithmetic: two cells per thread on the step grid (the caller
        // passes its blocks and width); FP64: one cell per thread
        if constexpr (sizeof(T) == 4)
            k_observe2<Q, S><<<nblocks, bx, 0, s>>>(a);
        else
            k_lattice<Q, T, S, kModeObserve><<<nblocks, bx, 0, s>>>(a);
        break;
    case kModeField:
        k_lattice<Q, T, S, kModeField><<<nblocks, bx, 0, s>>>(a);
        break;
    case kModeInit:
        k_init<Q, T, S, false><<<nblocks, bx, 0, s>>>(a);
        break;
    case kModeInitAcc:
        if constexpr (Storage<S>::kRef)
            k_init<Q, T, S, true><<<nblocks, bx, 0, s>>>(a);
        else
            return cudaErrorInvalidValue;
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int Q, typename T, typename S>
cudaError_t launch_batch_q(const void *table, const int *prefix, int n, int nblocks, int bx,
                           bool acc, cudaStream_t s)
{
    const StepArgs<T> *t = static_cast<const StepArgs<T> *>(table);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nblocks);
    cfg.blockDim = dim3((unsigned)bx);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (acc) {
        if constexpr (Storage<S>::kRef)
            return cudaLaunchKernelEx(&cfg, k_step_batch<Q, T, S, true>, t, prefix, n);
        else
            return cudaErrorInvalidValue;
    }
    return cudaLaunchKernelEx(&cfg, k_step_batch<Q, T, S, false>, t, prefix, n);
}

template <int Q, typename T>
cudaError_t launch_ref_q(const void *args, float *const enc[3], float *const dec[3], cudaStream_t s)
{
    const StepArgs<T> &a = *static_cast<const StepArgs<T> *>(args);
    const int total = (a.n_rows[kFluid] + 2 * a.n_rows[kSolid]) * Q;
    const int nb = (total + 255) / 256;
    k_ref_sum<Q, T><<<nb, 256, 0, s>>>(a, enc[0], enc[1], enc[2]);
    k_ref_dec<Q, T><<<nb, 256, 0, s>>>(a, enc[0], enc[1], enc[2], dec[0], dec[1], dec[2]);
    return cudaGetLastError();
}

}  // namespace klb
