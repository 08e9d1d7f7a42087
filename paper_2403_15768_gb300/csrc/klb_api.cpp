// C ABI of the KLB library (declared in include/klb.h): lattice creation in
// a caller-provided device buffer, couplings, initial state, time stepping,
// FP64 observables and host access to fields and state.

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "klb.h"
#include "klb_internal.h"

#ifndef KLB_BOUNDS
#define KLB_BOUNDS 0
#endif

using namespace klb;

// Host view of the time level of a lattice: steps taken, buffer holding the
// current state, and (reduced-precision storage) the reference generation of
// each buffer and whether the next step switches to refreshed references.
struct HostState {
    int64_t step = 0;
    int64_t since_reset = 0;  // steps since creation / init / set_state
    int cur = 0;              // state buffer holding g*(n-1)
    int gen_buf[2] = {0, 0};
    bool refresh_pending = false;
};

struct klb_lattice {
    klb_desc desc;
    std::vector<uint8_t> mask;
    Geometry geo;
    MemoryPlan plan;
    cudaStream_t stream = nullptr;
    char *base = nullptr;
    klb_couplings cp{0, 0, 0, 0, 0};
    double kT = 0.0;          // thermal fluctuations of the water (0: off)
    uint64_t seed = 0;
    HostState st;
    std::string err;
};

namespace {

thread_local std::string g_create_error;

klb_status fail(klb_lattice *L, klb_status st, const std::string &msg)
{
    if (L)
        L->err = msg;
    else
        g_create_error = msg;
    return st;
}

klb_status cuda_fail(klb_lattice *L, cudaError_t e, const char *what)
{
    return fail(L, KLB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define KLB_CUDA(L, call)                                         \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail((L), e_, #call);  \
    } while (0)

size_t pop_size(const klb_lattice *L) { return storage_bytes(L->desc.storage); }
size_t arith_size(const klb_lattice *L) { return L->desc.storage == KLB_FP64 ? 8 : 4; }
bool reduced(const klb_lattice *L) { return reduced_storage(L->desc.storage); }

void *dev(const klb_lattice *L, size_t off) { return L->base + off; }

// Lagged-velocity slot of step m (slots rotate with period 3).
int slot_of(int64_t m) { return (int)(((m % 3) + 3) % 3); }

// Kernel arguments for the time level `st` (the step about to run, or the
// one observed); the step kernel runs blocks of sbx threads.
template <typename T>
void fill_args_at(const klb_lattice *L, const HostState &st, int sbx, StepArgs<T> &a)
{
    const Geometry &g = L->geo;
    const MemoryPlan &p = L->plan;
    std::memset(&a, 0, sizeof a);
    const int64_t n = st.step;
    for (int s = 0; s < 3; ++s) {
        a.in[s] = dev(L, p.pop[st.cur][s]);
        a.out[s] = dev(L, p.pop[1 - st.cur][s]);
        a.in_prev[s] = dev(L, p.pop[1 - st.cur][s]);
    }
    if (reduced(L)) {
        for (int s = 0; s < 3; ++s) {
            a.dec_in[s] = (const float *)dev(L, p.ref_dec[st.gen_buf[st.cur]][s]);
            a.dec_prev[s] = (const float *)dev(L, p.ref_dec[st.gen_buf[1 - st.cur]][s]);
            a.enc_out[s] = (const float *)dev(L, p.ref_enc[st.gen_buf[st.cur]][s]);
        }
        a.scale = L->desc.storage == KLB_FP16_DEV ? kFp16Scale : 1.0f;
        a.inv_scale = 1.0f / a.scale;
        a.acc = (float *)dev(L, p.acc);
    } else {
        a.scale = a.inv_scale = 1.0f;
    }
    for (int c = 0; c < 2; ++c) {
        a.rows[c] = (const RowInfo *)dev(L, p.rows[c]);
        a.U0[c] = (T *)dev(L, p.U[slot_of(n)][c]);
        a.U1[c] = (const T *)dev(L, p.U[slot_of(n - 1)][c]);
        a.U2[c] = (const T *)dev(L, p.U[slot_of(n - 2)][c]);
        a.U3[c] = (const T *)dev(L, p.U[slot_of(n - 3)][c]);
        a.n_rows[c] = (int)g.rows[c].size();
        a.n_slots[c] = (int)g.slot_row[c].size();
    }
    a.nx = g.nx;
    a.nxp = g.nxp;
    a.nchunk = p.nchunk;
    a.nbw = (int)g.rows[kFluid].size() * a.nchunk;
    a.snchunk_w = step_chunks(g.nx, sbx, L->desc.storage, true);
    a.snchunk_s = step_chunks(g.nx, sbx, L->desc.storage, false);
    a.snbw = (int)g.rows[kFluid].size() * a.snchunk_w;
    a.nch32 = (g.nx + 31) / 32;
    a.nseg_w = (int)g.rows[kFluid].size() * a.nch32;
    const klb_desc &d = L->desc;
    a.rho0 = (T)d.rho0;
    a.om[0] = (T)(1.0 / d.tau_w);
    a.om[1] = (T)(1.0 / d.tau_e);
    a.om[2] = (T)(1.0 / d.tau_p);
    for (int k = 0; k < 3; ++k) a.G[k] = (T)d.G[k];
    a.g_we = (T)L->cp.g_we;
    a.g_wp = (T)L->cp.g_wp;
    a.g_ep = (T)L->cp.g_ep;
    a.g_ec = (T)L->cp.g_ec;
    a.g_pc = (T)L->cp.g_pc;
    a.q_p = (T)(d.phonon_eq == KLB_PHONON_WAVE ? 0.0 : 1.0);
    a.partials = (double *)dev(L, p.partials);
    a.residual_valid = st.since_reset >= 2;
    a.field = (T *)dev(L, p.field);
    const double om = 1.0 / d.tau_w;
    a.noise_amp = (T)(L->kT > 0.0 ? std::sqrt(3.0 * d.rho0 * L->kT * om * (2.0 - om)) : 0.0);
    a.key[0] = (uint32_t)(L->seed & 0xffffffffu);
    a.key[1] = (uint32_t)(L->seed >> 32);
    a.step_lo = (uint32_t)((uint64_t)n & 0xffffffffu);
    a.step_hi = (uint32_t)((uint64_t)n >> 32);
    a.bounds_err = (unsigned *)dev(L, p.bounds);
}

template <typename T>
void fill_args(const klb_lattice *L, StepArgs<T> &a)
{
    fill_args_at(L, L->st, L->plan.sbx, a);
}

// The host side of one step: encode generation of the output, whether the
// step accumulates x-sums for a reference refresh, and whether a refresh
// into that generation must run before it.
struct StepPlan {
    int outgen;
    bool acc;
    bool refresh;
};

StepPlan plan_step(const HostState &st, bool red)
{
    StepPlan sp;
    sp.outgen = st.gen_buf[st.cur];
    sp.refresh = red && st.refresh_pending;
    if (sp.refresh) sp.outgen = 1 - st.gen_buf[st.cur];
    sp.acc = red && (st.step + 1) % kRefEvery == 0;
    return sp;
}

void advance(HostState &st, const StepPlan &sp)
{
    st.gen_buf[1 - st.cur] = sp.outgen;
    st.cur = 1 - st.cur;
    ++st.step;
    ++st.since_reset;
    st.refresh_pending = sp.acc;
}

// Runs `body(args)` with arguments of the lattice's arithmetic type.
template <typename F>
cudaError_t with_args(const klb_lattice *L, F body)
{
    if (L->desc.storage == KLB_FP64) {
        StepArgs<double> a;
        fill_args(L, a);
        return body(&a);
    }
    StepArgs<float> a;
    fill_args(L, a);
    return body(&a);
}

// Sets the encode references of the next output buffer (generation gen).
void set_enc(const klb_lattice *L, void *args, int gen)
{
    if (!reduced(L)) return;
    StepArgs<float> *a = static_cast<StepArgs<float> *>(args);
    for (int s = 0; s < 3; ++s) a->enc_out[s] = (const float *)dev(L, L->plan.ref_enc[gen][s]);
}

// Reference refresh into generation gen from the x-sums of the last
// accumulating pass.
cudaError_t refresh_refs(const klb_lattice *L, int gen)
{
    float *enc[3], *dec[3];
    for (int s = 0; s < 3; ++s) {
        enc[s] = (float *)dev(L, L->plan.ref_enc[gen][s]);
        dec[s] = (float *)dev(L, L->plan.ref_dec[gen][s]);
    }
    return with_args(L, [&](void *a) { return launch_ref(L->geo.Q, L->desc.storage, a, enc, dec, L->stream); });
}

int nblocks(const klb_lattice *L) { return L->plan.nblocks_w + L->plan.nblocks_s; }

// Grid of the observation pass: with FP32 arithmetic two cells per thread on
// the step kernel's grid (at most nblocks(L) blocks, the size of the partial
// sums region), with FP64 one cell per thread.
int obs_blocks(const klb_lattice *L) { return L->desc.storage == KLB_FP64 ? nblocks(L) : L->plan.snblocks; }
int obs_bx(const klb_lattice *L) { return L->desc.storage == KLB_FP64 ? L->plan.bx : L->plan.sbx; }

// Species field index helpers: row class and row count of species s.
int cls_of(int s) { return s == 0 ? kFluid : kSolid; }

// Offset (elements) of species s in the field scratch [s][4][n_rows][nxp].
size_t field_offset(const klb_lattice *L, int s)
{
    const size_t nxp = L->geo.nxp, nrw = L->geo.rows[kFluid].size(),
                 nrs = L->geo.rows[kSolid].size();
    return s == 0 ? 0 : 4 * nrw * nxp + (s == 2 ? 4 * nrs * nxp : 0);
}

template <typename T>
void host_to_field(const klb_lattice *L, const double *drho, const double *u, std::vector<T> &f)
{
    const Geometry &g = L->geo;
    const size_t ncell = (size_t)g.nx * g.ny * g.nz, nxp = g.nxp;
    f.assign(L->plan.field_bytes / sizeof(T), T(0));
    for (int s = 0; s < 3; ++s) {
        const int c = cls_of(s);
        const size_t nr = g.rows[c].size(), fo = field_offset(L, s);
        for (size_t r = 0; r < nr; ++r) {
            const size_t cs = g.rows[c][r];
            for (int x = 0; x < g.nx; ++x) {
                const size_t cell = x + (size_t)g.nx * cs;
                f[fo + r * nxp + x] = drho ? (T)drho[s * ncell + cell] : T(0);
                for (int a = 0; a < 3; ++a)
                    f[fo + ((a + 1) * nr + r) * nxp + x] =
                        u ? (T)u[(s * 3 + a) * ncell + cell] : T(0);
            }
        }
    }
}

klb_status sync(klb_lattice *L)
{
    KLB_CUDA(L, cudaStreamSynchronize(L->stream));
    return KLB_OK;
}

template <typename T>
klb_status init_from_fields(klb_lattice *L, const double *drho, const double *u)
{
    std::vector<T> f;
    host_to_field<T>(L, drho, u, f);
    KLB_CUDA(L, cudaMemcpyAsync(dev(L, L->plan.field), f.data(), L->plan.field_bytes,
                                cudaMemcpyHostToDevice, L->stream));
    L->st.cur = 0;
    L->st.step = 0;
    L->st.since_reset = 0;
    L->st.gen_buf[0] = L->st.gen_buf[1] = 0;
    L->st.refresh_pending = false;
    const int slot0 = slot_of(0);
    auto init_pass = [&](int mode) {
        return with_args(L, [&](void *a) {
            StepArgs<T> *A = (StepArgs<T> *)a;
            for (int s = 0; s < 3; ++s) A->out[s] = dev(L, L->plan.pop[0][s]);
            for (int c = 0; c < 2; ++c) A->U0[c] = (T *)dev(L, L->plan.U[slot0][c]);
            set_enc(L, a, 0);
            return launch(L->geo.Q, L->desc.storage, a, mode, nblocks(L), L->plan.bx, L->stream);
        });
    };
    if (reduced(L)) {
        // References first: the x-averages of the initial equilibria.
        KLB_CUDA(L, init_pass(kModeInitAcc));
        KLB_CUDA(L, refresh_refs(L, 0));
    }
    KLB_CUDA(L, init_pass(kModeInit));
    for (int s = 0; s < 3; ++s)
        KLB_CUDA(L, cudaMemcpyAsync(dev(L, L->plan.pop[1][s]), dev(L, L->plan.pop[0][s]),
                                    L->plan.pop_bytes[s], cudaMemcpyDeviceToDevice, L->stream));
    for (int t = 0; t < 3; ++t)
        for (int c = 0; c < 2; ++c)
            if (t != slot0 && L->plan.U_bytes[c])
                KLB_CUDA(L, cudaMemcpyAsync(dev(L, L->plan.U[t][c]), dev(L, L->plan.U[slot0][c]),
                                            L->plan.U_bytes[c], cudaMemcpyDeviceToDevice, L->stream));
    return sync(L);
}

// Observables from the final sums (least squares u = A + B d^2 from its
// normal equations, means, residual, non-finite count); the one definition
// behind klb_observables and klb_observables_static.
klb_status finish_observables(klb_lattice *L, const double *S, klb_obs *out)
{
    const Geometry &g = L->geo;
    const double nan = std::numeric_limits<double>::quiet_NaN();
    std::memset(out, 0, sizeof *out);
    out->step = L->st.step;
    out->flow_rate = S[kSumUxFluid] / g.nx;
    out->d_wall = g.has_fit ? g.d_wall : nan;
    const double n = S[kSumFitN], s2 = S[kSumFitD2], s4 = S[kSumFitD4];
    const double su = S[kSumFitU], su2 = S[kSumFitUD2];
    const double det = n * s4 - s2 * s2;
    if (g.has_fit && n >= 2 && det != 0.0) {
        out->fit_B = (n * su2 - s2 * su) / det;
        out->fit_A = (su - out->fit_B * s2) / n;
        out->u_slip = out->fit_A + out->fit_B * g.d_wall * g.d_wall;
        out->dudn_wall = std::fabs(2.0 * out->fit_B * g.d_wall);
        out->slip_length = out->dudn_wall != 0.0 ? out->u_slip / out->dudn_wall
                                                 : std::numeric_limits<double>::infinity();
    } else {
        out->fit_A = out->fit_B = out->u_slip = out->dudn_wall = out->slip_length = nan;
    }
    out->u_wallrow_mean = S[kSumWallN] > 0 ? S[kSumWallU] / S[kSumWallN] : nan;
    const double ncells[3] = {(double)g.rows[kFluid].size() * g.nx,
                              (double)g.rows[kSolid].size() * g.nx,
                              (double)g.rows[kSolid].size() * g.nx};
    const double usum[3] = {S[kSumUxFluid], S[kSumUxE], S[kSumUxP]};
    for (int s = 0; s < 3; ++s) {
        out->mean_u[s] = usum[s] / ncells[s];
        out->momentum[s] = S[kSumMomW + s];
        out->mass[s] = S[kSumMassW + s];
    }
    out->residual = L->st.since_reset >= 2 ? S[kSumResidual] : nan;
    out->nonfinite = (int64_t)S[kSumNonfinite];
    out->clipped = (int64_t)S[kSumClipped];
    if (out->nonfinite > 0) return fail(L, KLB_EUNSTABLE, "non-finite density or velocity");
    if (out->clipped > 0)
        return fail(L, KLB_ERANGE,
                    std::to_string(out->clipped) +
                        " species-cells hold a population saturated at the 16-bit range (a difference "
                        "from the row's x-average beyond the representable range)");
    return KLB_OK;
}

bool finite5(const klb_couplings &c)
{
    return std::isfinite(c.g_we) && std::isfinite(c.g_wp) && std::isfinite(c.g_ep) &&
           std::isfinite(c.g_ec) && std::isfinite(c.g_pc);
}

}  // namespace

extern "C" {

size_t klb_lattice_bytes(const klb_desc *desc)
{
    if (!desc) return 0;
    Geometry g;
    std::string err;
    if (!build_geometry(*desc, g, err)) return 0;
    return plan_memory(g, desc->storage).total;
}

klb_status klb_lattice_info(const klb_desc *desc, klb_info *info)
{
    if (!desc || !info) return fail(nullptr, KLB_EINVAL, "null argument");
    Geometry g;
    std::string err;
    if (!build_geometry(*desc, g, err)) return fail(nullptr, KLB_EINVAL, err);
    std::memset(info, 0, sizeof *info);
    info->fluid_cs = (int64_t)g.rows[kFluid].size();
    info->solid_cs = (int64_t)g.rows[kSolid].size();
    info->species_cells[0] = info->fluid_cs * g.nx;
    info->species_cells[1] = info->species_cells[2] = info->solid_cs * g.nx;
    info->active_sites = (info->fluid_cs + info->solid_cs) * g.nx;
    for (int c = 0; c < 2; ++c) {
        info->iface_cs[c] = (int64_t)g.slot_row[c].size();
        info->max_faces[c] = g.max_faces[c];
    }
    info->d_wall = g.has_fit ? g.d_wall : std::numeric_limits<double>::quiet_NaN();
    info->bytes = plan_memory(g, desc->storage).total;
    return KLB_OK;
}

klb_status klb_create_lattice(const klb_desc *desc, void *dev_buf, size_t bytes, void *cuda_stream,
                              klb_lattice **out)
{
    if (!desc || !out) return fail(nullptr, KLB_EINVAL, "null argument");
    *out = nullptr;
    klb_lattice *L = new (std::nothrow) klb_lattice();
    if (!L) return fail(nullptr, KLB_ENOMEM, "host allocation failed");
    L->desc = *desc;
    if (desc->geom == KLB_GEOM_MASK && desc->mask && desc->ny > 0 && desc->nz > 0) {
        L->mask.assign(desc->mask, desc->mask + (size_t)desc->ny * desc->nz);
        L->desc.mask = L->mask.data();
    }
    std::string err;
    if (!build_geometry(L->desc, L->geo, err)) {
        delete L;
        return fail(nullptr, KLB_EINVAL, err);
    }
    L->plan = plan_memory(L->geo, L->desc.storage);
    if (!dev_buf || ((uintptr_t)dev_buf & 255u)) {
        delete L;
        return fail(nullptr, KLB_EINVAL, "dev_buf must be a 256-byte aligned device pointer");
    }
    if (bytes < L->plan.total) {
        delete L;
        return fail(nullptr, KLB_ENOMEM, "device buffer smaller than klb_lattice_bytes()");
    }
    L->base = (char *)dev_buf;
    L->stream = (cudaStream_t)cuda_stream;
    // Row tables, then a zero state.
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < 2 && e == cudaSuccess; ++c)
        e = cudaMemcpyAsync(dev(L, L->plan.rows[c]), L->geo.info[c].data(),
                            sizeof(RowInfo) * L->geo.info[c].size(), cudaMemcpyHostToDevice,
                            L->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dev(L, L->plan.bounds), 0, sizeof(unsigned), L->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
    if (e != cudaSuccess) {
        std::string m = std::string("uploading row tables: ") + cudaGetErrorString(e);
        delete L;
        return fail(nullptr, KLB_ECUDA, m);
    }
    klb_status st = klb_init_equilibrium(L, nullptr, nullptr);
    if (st != KLB_OK) {
        std::string m = L->err;
        delete L;
        return fail(nullptr, st, m);
    }
    *out = L;
    return KLB_OK;
}

klb_status klb_bounds_status(klb_lattice *L, uint32_t *site)
{
    if (!L || !site) return fail(L, KLB_EINVAL, "null argument");
    unsigned w = 0;
    KLB_CUDA(L, cudaMemcpyAsync(&w, dev(L, L->plan.bounds), sizeof w, cudaMemcpyDeviceToHost, L->stream));
    KLB_CUDA(L, cudaMemsetAsync(dev(L, L->plan.bounds), 0, sizeof w, L->stream));
    klb_status st = sync(L);
    if (st != KLB_OK) return st;
    *site = w;
    return KLB_OK;
}

int klb_bounds_checked(void) { return KLB_BOUNDS; }

klb_status klb_set_fluctuations(klb_lattice *L, double kT, uint64_t seed)
{
    if (!L) return fail(L, KLB_EINVAL, "null handle");
    if (!(kT >= 0.0) || !std::isfinite(kT)) return fail(L, KLB_EINVAL, "kT must be finite and >= 0");
    if (kT > 0.0 && reduced(L))
        return fail(L, KLB_EINVAL, "thermal fluctuations need FP32 or FP64 storage");
    L->kT = kT;
    L->seed = seed;
    return KLB_OK;
}

klb_status klb_set_couplings(klb_lattice *L, const klb_couplings *c)
{
    if (!L || !c) return fail(L, KLB_EINVAL, "null argument");
    if (!finite5(*c)) return fail(L, KLB_EINVAL, "non-finite coupling");
    // Stability of the lagged interface exchange (pair relaxation rate below
    // 4/3, Gershgorin over the cells): face-summed |gamma| below 0.6 rho0.
    const double sw = L->geo.max_faces[kFluid] * (std::fabs(c->g_we) + std::fabs(c->g_wp));
    const double ss = L->geo.max_faces[kSolid] * std::fmax(std::fabs(c->g_we), std::fabs(c->g_wp));
    if (std::fmax(sw, ss) >= 0.6 * L->desc.rho0)
        return fail(L, KLB_EINVAL, "interface couplings beyond the stability bound 0.6 rho0");
    // The co-located electron-phonon pair is implicit; only its matrix must stay regular.
    const double k = 0.5 * c->g_ep, a = L->desc.rho0 + k + 0.5 * c->g_ec,
                 b = L->desc.rho0 + k + 0.5 * c->g_pc;
    if (!(a > 0 && b > 0 && a * b - k * k > 0))
        return fail(L, KLB_EINVAL, "electron-phonon couplings make the implicit pair singular");
    L->cp = *c;
    return KLB_OK;
}

klb_status klb_init_equilibrium(klb_lattice *L, const double *drho, const double *u)
{
    if (!L) return fail(L, KLB_EINVAL, "null handle");
    return L->desc.storage == KLB_FP64 ? init_from_fields<double>(L, drho, u)
                                       : init_from_fields<float>(L, drho, u);
}

klb_status klb_step(klb_lattice *L, int64_t nsteps)
{
    if (!L) return fail(L, KLB_EINVAL, "null handle");
    if (nsteps < 0) return fail(L, KLB_EINVAL, "nsteps must be >= 0");
    for (int64_t n = 0; n < nsteps; ++n) {
        const StepPlan sp = plan_step(L->st, reduced(L));
        if (sp.refresh) {
            // Decode this step with the current references, encode its output
            // with references refreshed from the last step's x-averages.
            cudaError_t e = refresh_refs(L, sp.outgen);
            if (e != cudaSuccess) return cuda_fail(L, e, "reference refresh");
        }
        cudaError_t e = with_args(L, [&](void *a) {
            set_enc(L, a, sp.outgen);
            const int mode = sp.acc ? kModeStepAcc : (L->kT > 0.0 ? kModeStepNoise : kModeStep);
            return launch(L->geo.Q, L->desc.storage, a, mode, L->plan.snblocks, L->plan.sbx, L->stream);
        });
        if (e != cudaSuccess) return cuda_fail(L, e, "step kernel launch");
        advance(L->st, sp);
    }
    return KLB_OK;
}

}  // extern "C"

// Observation of many lattices with one synchronisation (the request loop):
// enqueue each lattice's pass and the copy of its sums to pinned host memory,
// synchronise the shared stream once, then finish each from its sums.
cudaError_t klb::observe_enqueue(klb_lattice *L, double *host_sums)
{
    cudaError_t e = with_args(L, [&](void *a) {
        return launch(L->geo.Q, L->desc.storage, a, kModeObserve, obs_blocks(L), obs_bx(L), L->stream);
    });
    if (e == cudaSuccess)
        e = launch_finalize((const double *)dev(L, L->plan.partials), obs_blocks(L), (double *)dev(L, L->plan.sums),
                            L->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_sums, dev(L, L->plan.sums), sizeof(double) * kNumSums, cudaMemcpyDeviceToHost,
                            L->stream);
    return e;
}

klb_status klb::observe_finish(klb_lattice *L, const double *host_sums, klb_obs *out)
{
    return finish_observables(L, host_sums, out);
}

extern "C" {

klb_status klb_observables(klb_lattice *L, klb_obs *out)
{
    if (!L || !out) return fail(L, KLB_EINVAL, "null argument");
    KLB_CUDA(L, with_args(L, [&](void *a) {
                 return launch(L->geo.Q, L->desc.storage, a, kModeObserve, obs_blocks(L),
                                    obs_bx(L), L->stream);
             }));
    KLB_CUDA(L, launch_finalize((const double *)dev(L, L->plan.partials), obs_blocks(L),
                                (double *)dev(L, L->plan.sums), L->stream));
    double S[kNumSums];
    KLB_CUDA(L, cudaMemcpyAsync(S, dev(L, L->plan.sums), sizeof S, cudaMemcpyDeviceToHost,
                                L->stream));
    klb_status st = sync(L);
    if (st != KLB_OK) return st;
    return finish_observables(L, S, out);
}

klb_status klb_observables_static(klb_lattice *L, klb_obs *out)
{
    if (!L || !out) return fail(L, KLB_EINVAL, "null argument");
    double *partials = nullptr, *sums = nullptr;
    size_t max_blocks = 0;
    KLB_CUDA(L, static_scratch(&partials, &sums, &max_blocks));
    if ((size_t)obs_blocks(L) > max_blocks)
        return fail(L, KLB_EINVAL,
                    "observation pass needs " + std::to_string(obs_blocks(L)) +
                        " blocks, more than the static scratch holds (KLB_STATIC_MAX_BLOCKS = " +
                        std::to_string(max_blocks) + ")");
    KLB_CUDA(L, with_args(L, [&](void *a) {
                 if (L->desc.storage == KLB_FP64)
                     static_cast<StepArgs<double> *>(a)->partials = partials;
                 else
                     static_cast<StepArgs<float> *>(a)->partials = partials;
                 return launch(L->geo.Q, L->desc.storage, a, kModeObserve, obs_blocks(L),
                                    obs_bx(L), L->stream);
             }));
    KLB_CUDA(L, launch_finalize(partials, obs_blocks(L), sums, L->stream));
    double S[kNumSums];
    KLB_CUDA(L, cudaMemcpyAsync(S, sums, sizeof S, cudaMemcpyDeviceToHost, L->stream));
    klb_status st = sync(L);
    if (st != KLB_OK) return st;
    return finish_observables(L, S, out);
}

klb_status klb_get_field(klb_lattice *L, double *drho, double *u)
{
    if (!L) return fail(L, KLB_EINVAL, "null handle");
    KLB_CUDA(L, with_args(L, [&](void *a) {
                 return launch(L->geo.Q, L->desc.storage, a, kModeField, nblocks(L),
                                    L->plan.bx, L->stream);
             }));
    const size_t ts = arith_size(L), nel = L->plan.field_bytes / ts;
    std::vector<double> f(nel);
    std::vector<char> raw(L->plan.field_bytes);
    KLB_CUDA(L, cudaMemcpyAsync(raw.data(), dev(L, L->plan.field), L->plan.field_bytes,
                                cudaMemcpyDeviceToHost, L->stream));
    klb_status st = sync(L);
    if (st != KLB_OK) return st;
    for (size_t k = 0; k < nel; ++k)
        f[k] = ts == 8 ? ((const double *)raw.data())[k] : (double)((const float *)raw.data())[k];
    const Geometry &g = L->geo;
    const size_t ncell = (size_t)g.nx * g.ny * g.nz, nxp = g.nxp;
    if (drho) std::memset(drho, 0, sizeof(double) * 3 * ncell);
    if (u) std::memset(u, 0, sizeof(double) * 9 * ncell);
    for (int s = 0; s < 3; ++s) {
        const int c = cls_of(s);
        const size_t nr = g.rows[c].size(), fo = field_offset(L, s);
        for (size_t r = 0; r < nr; ++r)
            for (int x = 0; x < g.nx; ++x) {
                const size_t cell = x + (size_t)g.nx * g.rows[c][r];
                if (drho) drho[s * ncell + cell] = f[fo + r * nxp + x];
                if (u)
                    for (int a = 0; a < 3; ++a)
                        u[(s * 3 + a) * ncell + cell] = f[fo + ((a + 1) * nr + r) * nxp + x];
            }
    }
    return KLB_OK;
}

klb_status klb_get_state(klb_lattice *L, double *gout, double *U1, double *U2)
{
    if (!L) return fail(L, KLB_EINVAL, "null handle");
    const Geometry &g = L->geo;
    const size_t ps = pop_size(L), ts = arith_size(L), ncell = (size_t)g.nx * g.ny * g.nz,
                 nxp = g.nxp;
    const int Q = g.Q;
    const bool red = reduced(L);
    const double inv = L->desc.storage == KLB_FP16_DEV ? 1.0 / kFp16Scale : 1.0;
    // Population value k of a downloaded buffer (reduced storage: the stored
    // difference, still to be scaled and shifted by its row reference).
    auto pop = [&](const std::vector<char> &raw, size_t k) -> double {
        switch (L->desc.storage) {
        case KLB_FP64:
            return ((const double *)raw.data())[k];
        case KLB_FP32:
            return ((const float *)raw.data())[k];
        case KLB_FP16_DEV:
            return (double)__half2float(((const __half *)raw.data())[k]);
        default:
            return (double)__bfloat162float(((const __nv_bfloat16 *)raw.data())[k]);
        }
    };
    auto rd = [&](const std::vector<char> &raw, size_t k) {
        return ts == 8 ? ((const double *)raw.data())[k] : (double)((const float *)raw.data())[k];
    };
    if (gout) {
        std::memset(gout, 0, sizeof(double) * 3 * Q * ncell);
        for (int s = 0; s < 3; ++s) {
            std::vector<char> raw(L->plan.pop_bytes[s]);
            KLB_CUDA(L, cudaMemcpyAsync(raw.data(), dev(L, L->plan.pop[L->st.cur][s]), raw.size(),
                                        cudaMemcpyDeviceToHost, L->stream));
            std::vector<float> ref;
            if (red) {
                ref.resize(L->plan.ref_bytes[s] / sizeof(float));
                KLB_CUDA(L, cudaMemcpyAsync(ref.data(), dev(L, L->plan.ref_enc[L->st.gen_buf[L->st.cur]][s]),
                                            L->plan.ref_bytes[s], cudaMemcpyDeviceToHost, L->stream));
            }
            klb_status st = sync(L);
            if (st != KLB_OK) return st;
            const int c = cls_of(s);
            const size_t nr = g.rows[c].size();
            for (int i = 0; i < Q; ++i)
                for (size_t r = 0; r < nr; ++r) {
                    const double shift = red ? (double)ref[r * kRefStride + i] : 0.0;
                    for (int x = 0; x < g.nx; ++x) {
                        double v = pop(raw, (i * nr + r) * nxp + x);
                        if (red) v = (double)(float)(v * inv + shift);
                        gout[((size_t)s * Q + i) * ncell + x + (size_t)g.nx * g.rows[c][r]] = v;
                    }
                }
        }
    }
    double *Uo[2] = {U1, U2};
    for (int t = 0; t < 2; ++t) {
        if (!Uo[t]) continue;
        std::memset(Uo[t], 0, sizeof(double) * 9 * ncell);
        const int slot = slot_of(L->st.step - 1 - t);
        for (int c = 0; c < 2; ++c) {
            const size_t ns = g.slot_row[c].size();
            if (!ns) continue;
            std::vector<char> raw(L->plan.U_bytes[c]);
            KLB_CUDA(L, cudaMemcpyAsync(raw.data(), dev(L, L->plan.U[slot][c]), raw.size(),
                                        cudaMemcpyDeviceToHost, L->stream));
            klb_status st = sync(L);
            if (st != KLB_OK) return st;
            for (size_t q = 0; q < ns; ++q) {
                const size_t cs = g.rows[c][g.slot_row[c][q]];
                for (int x = 0; x < g.nx; ++x) {
                    const size_t cell = x + (size_t)g.nx * cs;
                    for (int a = 0; a < 3; ++a) {
                        if (c == kFluid) {
                            Uo[t][a * ncell + cell] = rd(raw, (a * ns + q) * nxp + x);
                        } else {
                            Uo[t][(3 + a) * ncell + cell] = rd(raw, (a * ns + q) * nxp + x);
                            Uo[t][(6 + a) * ncell + cell] = rd(raw, ((a + 3) * ns + q) * nxp + x);
                        }
                    }
                }
            }
        }
    }
    (void)ps;
    return KLB_OK;
}

klb_status klb_set_state(klb_lattice *L, const double *gin, const double *U1, const double *U2,
                         int64_t step)
{
    if (!L || !gin || !U1 || !U2) return fail(L, KLB_EINVAL, "null argument");
    if (step < 0) return fail(L, KLB_EINVAL, "step must be >= 0");
    const Geometry &g = L->geo;
    const size_t ts = arith_size(L), ncell = (size_t)g.nx * g.ny * g.nz, nxp = g.nxp;
    const int Q = g.Q;
    const bool red = reduced(L);
    const double scale = L->desc.storage == KLB_FP16_DEV ? kFp16Scale : 1.0;
    auto sat = [](float v, float m) { return v > m ? m : (v < -m ? -m : v); };  // NaN passes
    auto put = [&](std::vector<char> &raw, size_t k, double v) {
        switch (L->desc.storage) {
        case KLB_FP64:
            ((double *)raw.data())[k] = v;
            break;
        case KLB_FP32:
            ((float *)raw.data())[k] = (float)v;
            break;
        case KLB_FP16_DEV:  // saturating, as the device encode
            ((__half *)raw.data())[k] = __float2half_rn(sat((float)v, 65504.0f));
            break;
        default:
            ((__nv_bfloat16 *)raw.data())[k] = __float2bfloat16_rn(sat((float)v, 3.38953139e38f));
            break;
        }
    };
    auto wr = [&](std::vector<char> &raw, size_t k, double v) {
        if (ts == 8)
            ((double *)raw.data())[k] = v;
        else
            ((float *)raw.data())[k] = (float)v;
    };
    KLB_CUDA(L, cudaStreamSynchronize(L->stream));
    L->st.cur = 0;
    L->st.step = step;
    L->st.since_reset = 0;
    L->st.gen_buf[0] = L->st.gen_buf[1] = 0;
    L->st.refresh_pending = false;
    std::vector<float> enc[3];
    for (int s = 0; s < 3; ++s) {
        const int c = cls_of(s);
        const size_t nr = g.rows[c].size();
        if (red) {
            // Reference of each (row, direction): the x-average of the state.
            enc[s].assign(nr * kRefStride, 0.f);
            for (int i = 0; i < Q; ++i)
                for (size_t r = 0; r < nr; ++r) {
                    double sum = 0.0;
                    for (int x = 0; x < g.nx; ++x)
                        sum += gin[((size_t)s * Q + i) * ncell + x + (size_t)g.nx * g.rows[c][r]];
                    enc[s][r * kRefStride + i] = (float)(sum / g.nx);
                }
        }
        std::vector<char> raw(L->plan.pop_bytes[s], 0);
        for (int i = 0; i < Q; ++i)
            for (size_t r = 0; r < nr; ++r) {
                const float ref = red ? enc[s][r * kRefStride + i] : 0.f;
                for (int x = 0; x < g.nx; ++x) {
                    const double v = gin[((size_t)s * Q + i) * ncell + x + (size_t)g.nx * g.rows[c][r]];
                    put(raw, (i * nr + r) * nxp + x, red ? ((float)v - ref) * (float)scale : v);
                }
            }
        for (int b = 0; b < 2; ++b)
            KLB_CUDA(L, cudaMemcpy(dev(L, L->plan.pop[b][s]), raw.data(), raw.size(),
                                   cudaMemcpyHostToDevice));
    }
    if (red) {
        for (int s = 0; s < 3; ++s) {
            const int c = cls_of(s);
            const size_t nr = g.rows[c].size();
            std::vector<float> dec(nr * kRefStride, 0.f);
            for (size_t r = 0; r < nr; ++r)
                for (int i = 0; i < Q; ++i) {
                    const long q = g.info[c][r].src[i] / (g.nxp / kRowAlign);  // sdir * nr + srow
                    const long sdir = q / (long)nr, srow = q - sdir * (long)nr;
                    dec[r * kRefStride + i] = enc[s][srow * kRefStride + sdir];
                }
            KLB_CUDA(L, cudaMemcpy(dev(L, L->plan.ref_enc[0][s]), enc[s].data(), L->plan.ref_bytes[s],
                                   cudaMemcpyHostToDevice));
            KLB_CUDA(L, cudaMemcpy(dev(L, L->plan.ref_dec[0][s]), dec.data(), L->plan.ref_bytes[s],
                                   cudaMemcpyHostToDevice));
        }
    }
    const double *Ui[3] = {U1, U2, U2};  // u(n-1), u(n-2); u(n-3) unknown: reuse u(n-2)
    for (int t = 0; t < 3; ++t) {
        const int slot = slot_of(step - 1 - t);
        for (int c = 0; c < 2; ++c) {
            const size_t ns = g.slot_row[c].size();
            if (!ns) continue;
            std::vector<char> raw(L->plan.U_bytes[c], 0);
            for (size_t q = 0; q < ns; ++q) {
                const size_t cs = g.rows[c][g.slot_row[c][q]];
                for (int x = 0; x < g.nx; ++x) {
                    const size_t cell = x + (size_t)g.nx * cs;
                    for (int a = 0; a < 3; ++a) {
                        if (c == kFluid) {
                            wr(raw, (a * ns + q) * nxp + x, Ui[t][a * ncell + cell]);
                        } else {
                            wr(raw, (a * ns + q) * nxp + x, Ui[t][(3 + a) * ncell + cell]);
                            wr(raw, ((a + 3) * ns + q) * nxp + x, Ui[t][(6 + a) * ncell + cell]);
                        }
                    }
                }
            }
            KLB_CUDA(L, cudaMemcpy(dev(L, L->plan.U[slot][c]), raw.data(), raw.size(),
                                   cudaMemcpyHostToDevice));
        }
    }
    return KLB_OK;
}

int64_t klb_get_step(const klb_lattice *L) { return L ? L->st.step : -1; }

int64_t klb_species_cells(const klb_lattice *L, int species)
{
    if (!L || species < 0 || species > 2) return -1;
    return (int64_t)L->geo.rows[cls_of(species)].size() * L->geo.nx;
}

klb_status klb_destroy(klb_lattice *L)
{
    if (!L) return KLB_OK;
    cudaError_t e = cudaStreamSynchronize(L->stream);
    delete L;
    if (e != cudaSuccess) {
        g_create_error = std::string("klb_destroy: ") + cudaGetErrorString(e);
        return KLB_ECUDA;
    }
    return KLB_OK;
}

const char *klb_last_error(const klb_lattice *L)
{
    return L ? L->err.c_str() : g_create_error.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches

struct klb_batch {
    std::vector<klb_lattice *> mem;
    cudaStream_t user = nullptr;  // the members' stream
    cudaStream_t stream = nullptr;  // the batch's own stream (graph capture)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    char *base = nullptr;
    size_t bytes = 0;
    int Q = 19, storage = KLB_FP32;
    int period = 6;
    int width = kBlockX;
    int nblocks = 0;
    size_t args_size = 0, table_off = 0, prefix_off = 0, reps_off = 0;
    std::vector<StepPlan> plans;  // per (phase, member)
    std::vector<char> acc;        // per phase: some member accumulates x-sums
    std::vector<int64_t> base_step;  // members' steps at phase 0
    std::vector<HostState> base_state;  // members' time levels at phase 0
    int64_t phase = 0;               // steps taken since phase 0
    cudaGraphExec_t graph = nullptr;
    std::string err;
};

namespace {

klb_status bfail(klb_batch *B, klb_status st, const std::string &msg)
{
    B->err = msg;
    return st;
}

#define KLB_BCUDA(B, call)                                                                  \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return bfail((B), KLB_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int batch_period(int storage) { return reduced_storage(storage) ? 6 * 2 * kRefEvery : 6; }

size_t args_size(int storage) { return storage == KLB_FP64 ? sizeof(StepArgs<double>) : sizeof(StepArgs<float>); }

// Batch buffer: argument tables [phase][member], block prefix, period count.
size_t batch_layout(int n, int storage, size_t *table_off, size_t *prefix_off, size_t *reps_off)
{
    const size_t tb = (size_t)batch_period(storage) * n * args_size(storage);
    *table_off = 0;
    *prefix_off = (tb + 255) / 256 * 256;
    *reps_off = *prefix_off + ((size_t)(n + 1) * sizeof(int) + 255) / 256 * 256;
    return *reps_off + 256;
}

void destroy_graph(klb_batch *B)
{
    if (B->graph) cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
}

// Per-phase argument tables for block width `width`, from each member's own
// time level now (phase 0), the block prefix, and the phase plans.  Every
// member's step pattern repeats after the batch period whatever its step
// count, so members may stand at different time levels.  A launch
// accumulates reference x-sums when any member needs them; the x-sums are
// stored, not added, so an extra pass leaves the other members' refreshes
// unchanged.
klb_status build_tables(klb_batch *B, int width)
{
    const int n = (int)B->mem.size(), P = B->period;
    std::vector<char> host((size_t)P * n * B->args_size);
    std::vector<int> prefix(n + 1, 0);
    B->plans.assign((size_t)P * n, StepPlan{0, false, false});
    B->acc.assign(P, 0);
    for (int m = 0; m < n; ++m) {
        const klb_lattice *L = B->mem[m];
        HostState st = L->st;
        for (int k = 0; k < P; ++k) {
            const StepPlan sp = plan_step(st, reduced(L));
            B->plans[(size_t)k * n + m] = sp;
            B->acc[k] |= (char)sp.acc;
            char *slot = host.data() + ((size_t)k * n + m) * B->args_size;
            const uint32_t *reps = (const uint32_t *)(B->base + B->reps_off);
            if (B->storage == KLB_FP64) {
                StepArgs<double> a;
                fill_args_at(L, st, width, a);
                a.step_reps = reps;
                a.step_period = P;
                std::memcpy(slot, &a, sizeof a);
            } else {
                StepArgs<float> a;
                fill_args_at(L, st, width, a);
                a.step_reps = reps;
                a.step_period = P;
                if (reduced(L))
                    for (int s = 0; s < 3; ++s) a.enc_out[s] = (const float *)dev(L, L->plan.ref_enc[sp.outgen][s]);
                std::memcpy(slot, &a, sizeof a);
            }
            advance(st, sp);
        }
        const int sto = L->desc.storage;
        prefix[m + 1] = prefix[m] +
                        step_chunks(L->geo.nx, width, sto, true) * (int)L->geo.rows[kFluid].size() +
                        step_chunks(L->geo.nx, width, sto, false) * (int)L->geo.rows[kSolid].size();
    }
    KLB_BCUDA(B, cudaStreamSynchronize(B->stream));
    KLB_BCUDA(B, cudaMemcpy(B->base + B->table_off, host.data(), host.size(), cudaMemcpyHostToDevice));
    KLB_BCUDA(B, cudaMemcpy(B->base + B->prefix_off, prefix.data(), prefix.size() * sizeof(int),
                            cudaMemcpyHostToDevice));
    KLB_BCUDA(B, cudaMemset(B->base + B->reps_off, 0, sizeof(uint32_t)));
    B->width = width;
    B->nblocks = prefix[n];
    B->phase = 0;
    B->base_step.resize(n);
    B->base_state.resize(n);
    for (int m = 0; m < n; ++m) {
        B->base_step[m] = B->mem[m]->st.step;
        B->base_state[m] = B->mem[m]->st;
    }
    destroy_graph(B);
    return KLB_OK;
}

// One phase of the batch on its stream: reference refreshes due before the
// step, then the batched step kernel.
cudaError_t launch_phase(klb_batch *B, int k)
{
    const size_t n = B->mem.size();
    for (size_t m = 0; m < n; ++m) {
        const StepPlan &sp = B->plans[k * n + m];
        if (!sp.refresh) continue;
        klb_lattice *L = B->mem[m];
        cudaStream_t keep = L->stream;
        L->stream = B->stream;
        cudaError_t e = refresh_refs(L, sp.outgen);
        L->stream = keep;
        if (e != cudaSuccess) return e;
    }
    const char *table = B->base + B->table_off + (size_t)k * n * B->args_size;
    cudaError_t e = launch_batch(B->Q, B->storage, table, (const int *)(B->base + B->prefix_off), (int)n,
                                 B->nblocks, B->width, B->acc[k] != 0, B->stream);
    if (e == cudaSuccess && k == B->period - 1) e = launch_count_period((uint32_t *)(B->base + B->reps_off), B->stream);
    return e;
}

klb_status capture_graph(klb_batch *B)
{
    destroy_graph(B);
    cudaGraph_t g = nullptr;
    KLB_BCUDA(B, cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < B->period && e == cudaSuccess; ++k) e = launch_phase(B, k);
    cudaError_t e2 = cudaStreamEndCapture(B->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(B, KLB_ECUDA, std::string("graph capture: ") +
                                       cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&B->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        B->graph = nullptr;
        return bfail(B, KLB_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    return KLB_OK;
}

bool in_phase(const klb_batch *B)
{
    for (size_t m = 0; m < B->mem.size(); ++m)
        if (B->mem[m]->st.step != B->base_step[m] + B->phase) return false;
    return true;
}

// Whether every member stands where the tables' phase 0 assumed.  The step
// pattern repeats after a period from any time level but one: right after
// an initialisation of 16-bit storage no reference refresh is pending at a
// multiple of the refresh interval, where one is pending in every later
// period.
bool tables_repeat(const klb_batch *B)
{
    for (size_t m = 0; m < B->mem.size(); ++m) {
        const HostState &a = B->mem[m]->st, &b = B->base_state[m];
        if (a.cur != b.cur || a.gen_buf[0] != b.gen_buf[0] || a.gen_buf[1] != b.gen_buf[1] ||
            a.refresh_pending != b.refresh_pending)
            return false;
    }
    return true;
}

// Runs nsteps phases on the batch stream, replaying the graph for whole
// periods; advances every member's host state.  At the start of each later
// period the tables are checked against the members' time levels and built
// again if they no longer describe it.
klb_status run_steps(klb_batch *B, int64_t nsteps, bool use_graph)
{
    while (nsteps > 0) {
        if (B->phase > 0 && B->phase % B->period == 0 && !tables_repeat(B)) {
            klb_status st = build_tables(B, B->width);
            if (st != KLB_OK) return st;
        }
        const int k = (int)(B->phase % B->period);
        if (use_graph && k == 0 && nsteps >= B->period) {
            if (!B->graph) {
                klb_status st = capture_graph(B);
                if (st != KLB_OK) return st;
            }
            KLB_BCUDA(B, cudaGraphLaunch(B->graph, B->stream));
            for (klb_lattice *L : B->mem) {
                HostState &h = L->st;
                for (int j = 0; j < B->period; ++j) advance(h, plan_step(h, reduced(L)));
            }
            B->phase += B->period;
            nsteps -= B->period;
            continue;
        }
        KLB_BCUDA(B, launch_phase(B, k));
        for (klb_lattice *L : B->mem) advance(L->st, plan_step(L->st, reduced(L)));
        ++B->phase;
        --nsteps;
    }
    return KLB_OK;
}

}  // namespace

size_t klb::batch_table_bytes(int storage, int n)
{
    size_t t, p, r;
    return n < 1 ? 0 : batch_layout(n, storage, &t, &p, &r);
}

extern "C" {

size_t klb_batch_bytes(klb_lattice *const *members, int n)
{
    if (!members || n < 1 || !members[0]) return 0;
    size_t t, p, r;
    return batch_layout(n, members[0]->desc.storage, &t, &p, &r);
}

klb_status klb_batch_create(klb_lattice *const *members, int n, void *dev_buf, size_t bytes,
                            klb_batch **out)
{
    if (!out) return fail(nullptr, KLB_EINVAL, "null argument");
    *out = nullptr;
    if (!members || n < 1) return fail(nullptr, KLB_EINVAL, "a batch needs at least one member");
    for (int m = 0; m < n; ++m) {
        const klb_lattice *L = members[m];
        if (!L) return fail(nullptr, KLB_EINVAL, "null member");
        if (L->geo.Q != members[0]->geo.Q || L->desc.storage != members[0]->desc.storage)
            return fail(nullptr, KLB_EINVAL, "batch members must share lattice kind and storage");
        if (L->stream != members[0]->stream)
            return fail(nullptr, KLB_EINVAL, "batch members must share one CUDA stream");
        for (int k = 0; k < m; ++k)
            if (members[k] == L) return fail(nullptr, KLB_EINVAL, "a lattice appears twice in the batch");
        if (L->kT > 0.0)
            return fail(nullptr, KLB_EINVAL, "lattices with thermal fluctuations cannot be batched");
    }
    klb_batch *B = new (std::nothrow) klb_batch();
    if (!B) return fail(nullptr, KLB_ENOMEM, "host allocation failed");
    B->mem.assign(members, members + n);
    B->Q = members[0]->geo.Q;
    B->storage = members[0]->desc.storage;
    B->period = batch_period(B->storage);
    B->args_size = args_size(B->storage);
    const size_t need = batch_layout(n, B->storage, &B->table_off, &B->prefix_off, &B->reps_off);
    if (!dev_buf || ((uintptr_t)dev_buf & 255u)) {
        delete B;
        return fail(nullptr, KLB_EINVAL, "dev_buf must be a 256-byte aligned device pointer");
    }
    if (bytes < need) {
        delete B;
        return fail(nullptr, KLB_ENOMEM, "device buffer smaller than klb_batch_bytes()");
    }
    B->base = (char *)dev_buf;
    B->bytes = bytes;
    B->user = members[0]->stream;
    cudaError_t e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->user);
    if (e != cudaSuccess) {
        std::string m = std::string("batch setup: ") + cudaGetErrorString(e);
        klb_batch_destroy(B);
        return fail(nullptr, KLB_ECUDA, m);
    }
    int w = kBlockX;
    for (klb_lattice *L : B->mem) w = std::min(w, L->plan.sbx);
    klb_status st = build_tables(B, w);
    if (st != KLB_OK) {
        std::string m = B->err;
        klb_batch_destroy(B);
        return fail(nullptr, st, m);
    }
    *out = B;
    return KLB_OK;
}

klb_status klb_batch_step(klb_batch *B, int64_t nsteps)
{
    if (!B) return KLB_EINVAL;
    if (nsteps < 0) return bfail(B, KLB_EINVAL, "nsteps must be >= 0");
    if (!in_phase(B))
        return bfail(B, KLB_ESTATE, "a member was stepped outside the batch; form the batch again");
    KLB_BCUDA(B, cudaEventRecord(B->ev_in, B->user));
    KLB_BCUDA(B, cudaStreamWaitEvent(B->stream, B->ev_in, 0));
    klb_status st = run_steps(B, nsteps, true);
    KLB_BCUDA(B, cudaEventRecord(B->ev_out, B->stream));
    KLB_BCUDA(B, cudaStreamWaitEvent(B->user, B->ev_out, 0));
    return st;
}

klb_status klb_batch_autotune(klb_batch *B, int steps_per_candidate, int *width)
{
    if (!B) return KLB_EINVAL;
    if (steps_per_candidate < 1) return bfail(B, KLB_EINVAL, "steps_per_candidate must be >= 1");
    if (!in_phase(B))
        return bfail(B, KLB_ESTATE, "a member was stepped outside the batch; form the batch again");
    KLB_BCUDA(B, cudaStreamSynchronize(B->user));
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t ce = cudaEventCreate(&t0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&t1);
    if (ce != cudaSuccess) {
        if (t0) cudaEventDestroy(t0);
        return bfail(B, KLB_ECUDA, std::string("autotune events: ") + cudaGetErrorString(ce));
    }
    const int cand[3] = {32, 64, 128};
    int best = B->width;
    float best_ms = 1e30f;
    klb_status st = KLB_OK;
    for (int c = 0; c < 3 && st == KLB_OK; ++c) {
        st = build_tables(B, cand[c]);
        if (st != KLB_OK) break;
        st = run_steps(B, 1, false);  // warm-up
        if (st != KLB_OK) break;
        if (cudaEventRecord(t0, B->stream) != cudaSuccess) {
            st = bfail(B, KLB_ECUDA, "autotune timing");
            break;
        }
        st = run_steps(B, steps_per_candidate, false);
        if (st != KLB_OK) break;
        float ms = 0.f;
        if (cudaEventRecord(t1, B->stream) != cudaSuccess || cudaEventSynchronize(t1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, t0, t1) != cudaSuccess)
            st = bfail(B, KLB_ECUDA, "autotune timing");
        if (st == KLB_OK && ms < best_ms) {
            best_ms = ms;
            best = cand[c];
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (st != KLB_OK) return st;
    st = build_tables(B, best);
    if (width) *width = best;
    return st;
}

int klb_batch_width(const klb_batch *B) { return B ? B->width : 0; }
int64_t klb_batch_blocks(const klb_batch *B) { return B ? B->nblocks : 0; }

klb_status klb_batch_destroy(klb_batch *B)
{
    if (!B) return KLB_OK;
    if (B->stream) cudaStreamSynchronize(B->stream);
    destroy_graph(B);
    if (B->ev_in) cudaEventDestroy(B->ev_in);
    if (B->ev_out) cudaEventDestroy(B->ev_out);
    if (B->stream) cudaStreamDestroy(B->stream);
    delete B;
    return KLB_OK;
}

const char *klb_batch_last_error(const klb_batch *B) { return B ? B->err.c_str() : ""; }

}  // extern "C"
