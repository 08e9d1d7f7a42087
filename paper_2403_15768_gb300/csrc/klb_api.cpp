// C ABI of the KLB library (declared in include/klb.h): lattice creation in
// a caller-provided device buffer, couplings, initial state, time stepping,
// FP64 observables and host access to fields and state.

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

using namespace klb;

struct klb_lattice {
    klb_desc desc;
    std::vector<uint8_t> mask;
    Geometry geo;
    MemoryPlan plan;
    cudaStream_t stream = nullptr;
    char *base = nullptr;
    klb_couplings cp{0, 0, 0, 0, 0};
    int64_t step = 0;
    int64_t since_reset = 0;  // steps since creation / init / set_state
    int cur = 0;              // state buffer holding g*(n-1)
    // Reduced-precision storage: reference generation each state buffer is
    // encoded with, and whether the next step switches to refreshed references.
    int gen_buf[2] = {0, 0};
    bool refresh_pending = false;
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

template <typename T>
void fill_args(const klb_lattice *L, StepArgs<T> &a)
{
    const Geometry &g = L->geo;
    const MemoryPlan &p = L->plan;
    std::memset(&a, 0, sizeof a);
    const int n = (int)L->step;  // the step about to run / being observed
    for (int s = 0; s < 3; ++s) {
        a.in[s] = dev(L, p.pop[L->cur][s]);
        a.out[s] = dev(L, p.pop[1 - L->cur][s]);
        a.in_prev[s] = dev(L, p.pop[1 - L->cur][s]);
    }
    if (reduced(L)) {
        for (int s = 0; s < 3; ++s) {
            a.dec_in[s] = (const float *)dev(L, p.ref_dec[L->gen_buf[L->cur]][s]);
            a.dec_prev[s] = (const float *)dev(L, p.ref_dec[L->gen_buf[1 - L->cur]][s]);
            a.enc_out[s] = (const float *)dev(L, p.ref_enc[L->gen_buf[L->cur]][s]);
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
    a.nbw = p.nblocks_w;
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
    a.partials = (double *)dev(L, p.partials);
    a.residual_valid = L->since_reset >= 2;
    a.field = (T *)dev(L, p.field);
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
    L->cur = 0;
    L->step = 0;
    L->since_reset = 0;
    L->gen_buf[0] = L->gen_buf[1] = 0;
    L->refresh_pending = false;
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

// Observables from the final sums, for klb_observables_static (the same
// definitions as klb_observables).
klb_status finish_observables(klb_lattice *L, const double *S, klb_obs *out)
{
    const Geometry &g = L->geo;
    const double nan = std::numeric_limits<double>::quiet_NaN();
    std::memset(out, 0, sizeof *out);
    out->step = L->step;
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
    out->residual = L->since_reset >= 2 ? S[kSumResidual] : nan;
    out->nonfinite = (int64_t)S[kSumNonfinite];
    if (out->nonfinite > 0) return fail(L, KLB_EUNSTABLE, "non-finite density or velocity");
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
        int outgen = L->gen_buf[L->cur];
        if (reduced(L) && L->refresh_pending) {
            // Decode this step with the current references, encode its output
            // with references refreshed from the last step's x-averages.
            outgen = 1 - L->gen_buf[L->cur];
            cudaError_t e = refresh_refs(L, outgen);
            if (e != cudaSuccess) return cuda_fail(L, e, "reference refresh");
            L->refresh_pending = false;
        }
        const bool acc = reduced(L) && (L->step + 1) % kRefEvery == 0;
        cudaError_t e = with_args(L, [&](void *a) {
            set_enc(L, a, outgen);
            return launch(L->geo.Q, L->desc.storage, a, acc ? kModeStepAcc : kModeStep, nblocks(L),
                          L->plan.bx, L->stream);
        });
        if (e != cudaSuccess) return cuda_fail(L, e, "step kernel launch");
        L->gen_buf[1 - L->cur] = outgen;
        L->cur = 1 - L->cur;
        ++L->step;
        ++L->since_reset;
        if (acc) L->refresh_pending = true;
    }
    return KLB_OK;
}

klb_status klb_observables(klb_lattice *L, klb_obs *out)
{
    if (!L || !out) return fail(L, KLB_EINVAL, "null argument");
    KLB_CUDA(L, with_args(L, [&](void *a) {
                 return launch(L->geo.Q, L->desc.storage, a, kModeObserve, nblocks(L),
                                    L->plan.bx, L->stream);
             }));
    KLB_CUDA(L, launch_finalize((const double *)dev(L, L->plan.partials), nblocks(L),
                                (double *)dev(L, L->plan.sums), L->stream));
    double S[kNumSums];
    KLB_CUDA(L, cudaMemcpyAsync(S, dev(L, L->plan.sums), sizeof S, cudaMemcpyDeviceToHost,
                                L->stream));
    klb_status st = sync(L);
    if (st != KLB_OK) return st;

    const Geometry &g = L->geo;
    const double nan = std::numeric_limits<double>::quiet_NaN();
    std::memset(out, 0, sizeof *out);
    out->step = L->step;
    out->flow_rate = S[kSumUxFluid] / g.nx;
    out->d_wall = g.has_fit ? g.d_wall : nan;
    // Least squares u = A + B d^2 from its normal equations.
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
    out->residual = L->since_reset >= 2 ? S[kSumResidual] : nan;
    out->nonfinite = (int64_t)S[kSumNonfinite];
    if (out->nonfinite > 0) return fail(L, KLB_EUNSTABLE, "non-finite density or velocity");
    return KLB_OK;
}

klb_status klb_observables_static(klb_lattice *L, klb_obs *out)
{
    if (!L || !out) return fail(L, KLB_EINVAL, "null argument");
    double *partials = nullptr, *sums = nullptr;
    size_t max_blocks = 0;
    KLB_CUDA(L, static_scratch(&partials, &sums, &max_blocks));
    if ((size_t)nblocks(L) > max_blocks)
        return fail(L, KLB_EINVAL,
                    "observation pass needs " + std::to_string(nblocks(L)) +
                        " blocks, more than the static scratch holds (KLB_STATIC_MAX_BLOCKS = " +
                        std::to_string(max_blocks) + ")");
    KLB_CUDA(L, with_args(L, [&](void *a) {
                 if (L->desc.storage == KLB_FP64)
                     static_cast<StepArgs<double> *>(a)->partials = partials;
                 else
                     static_cast<StepArgs<float> *>(a)->partials = partials;
                 return launch(L->geo.Q, L->desc.storage, a, kModeObserve, nblocks(L),
                                    L->plan.bx, L->stream);
             }));
    KLB_CUDA(L, launch_finalize(partials, nblocks(L), sums, L->stream));
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
            KLB_CUDA(L, cudaMemcpyAsync(raw.data(), dev(L, L->plan.pop[L->cur][s]), raw.size(),
                                        cudaMemcpyDeviceToHost, L->stream));
            std::vector<float> ref;
            if (red) {
                ref.resize(L->plan.ref_bytes[s] / sizeof(float));
                KLB_CUDA(L, cudaMemcpyAsync(ref.data(), dev(L, L->plan.ref_enc[L->gen_buf[L->cur]][s]),
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
        const int slot = slot_of(L->step - 1 - t);
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
    auto put = [&](std::vector<char> &raw, size_t k, double v) {
        switch (L->desc.storage) {
        case KLB_FP64:
            ((double *)raw.data())[k] = v;
            break;
        case KLB_FP32:
            ((float *)raw.data())[k] = (float)v;
            break;
        case KLB_FP16_DEV:
            ((__half *)raw.data())[k] = __float2half_rn((float)v);
            break;
        default:
            ((__nv_bfloat16 *)raw.data())[k] = __float2bfloat16_rn((float)v);
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
    L->cur = 0;
    L->step = step;
    L->since_reset = 0;
    L->gen_buf[0] = L->gen_buf[1] = 0;
    L->refresh_pending = false;
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
                    const long q = g.info[c][r].src[i] / g.nxp;  // sdir * nr + srow
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

int64_t klb_get_step(const klb_lattice *L) { return L ? L->step : -1; }

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
