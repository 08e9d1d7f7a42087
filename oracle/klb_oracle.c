/*
 * klb_oracle.c -- plain, slow FP64 CPU oracle of one time step of the
 * three-species Keldysh-lattice Boltzmann (KLB) scheme: water ("hydron")
 * populations h_i on fluid cells, electron e_i and phonon p_i populations on
 * solid cells (Sec. 4 of the paper).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled, loaded and called only by
 * the tests, by the smoke check and by the CPU-baseline leg of the benchmark.
 * The product library never includes, links or calls it, and it shares no
 * code, table or helper with the CUDA path.
 *
 * Storage: dense boxes, x fastest.  Cell (x,y,z) has index
 * x + nx*(y + ny*z).  Population i of a species lives at [i*ncell + cell].
 * Populations are kept as deviations g_i = f_i - w_i*rho0 from the rest state.
 * Cells that do not carry a species hold zeros for it and are never read.
 *
 * One step, in this order (the state is the post-collision deviation g*):
 *   1. pull-stream, with the boundary rules of Sec. 4.2 (Eqs. 19-24) read as
 *      described at stream_source();
 *   2. moments  drho = sum_i g_i,  j = sum_i c_i g_i;
 *   3. interface friction at fluid/solid faces, antisymmetric as in Eq. 27
 *      (water side Eq. 5, electron side Eq. 11, phonon side Eq. 15), from the
 *      lagged velocities Ubar = (u(n-1) + u(n-2))/2 of both partners (see
 *      interface_velocity());
 *   4. co-located electron-phonon friction and crystal sinks (Eqs. 12, 13, 16),
 *      trapezoidal in time, solved exactly per cell; water velocity with the
 *      pressure drive of Eq. 2 as a uniform body force;
 *   5. U2 := U, U := u for the next step;
 *   6. BGK collision with Guo forcing;
 *   7. optionally, thermal fluctuations of the water (see thermal_noise()).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { T_VOID = 0, T_FLUID = 1, T_SOLID = 2 };
enum { SW = 0, SE = 1, SP = 2 }; /* species: water, electron, phonon */

typedef struct {
    int Q;
    int c[19][3];
    double w[19];
    int opp[19];

    int nx, ny, nz;
    int periodic_y, periodic_z;
    unsigned char *cs_type; /* ny*nz cross-section map, index y + ny*z */
    long ncell;

    double tau[3];
    double rho0;
    double G[3];
    double g_we, g_wp, g_ep, g_ec, g_pc;
    int iface_bounceback;

    /* stream_source() evaluated once per (species, cross-section cell,
     * direction): the geometry does not depend on x, so the source of the
     * link at (x,y,z) is (x + sdx, sy, sz), population sdir.  -1: no species. */
    int *sdx[3], *sy[3], *sz[3], *sdir[3];

    double *gs[3];   /* post-collision deviations (the state)          */
    double *U[3];    /* velocity of step n-1, [a*ncell + cell]         */
    double *U2[3];   /* velocity of step n-2                           */
    double *g[3];    /* streamed (pre-collision) deviations            */
    double *drho[3]; /* density deviation of the current step          */
    double *u[3];    /* velocity of the current step, [a*ncell + cell] */
    double *F[3];    /* total force density of the current step        */
    long step;
    int phonon_wave; /* 1: phonons follow the damped wave equation of Sec. 3.4 */
    double kT;       /* thermal energy of the water fluctuations (0: off) */
    uint32_t key[2]; /* generator key (seed)                              */
} kor_t;

/* ------------------------------------------------------------------ */
/* Lattices.  D2Q9 in the paper's numbering (Sec. 4.2): 0 rest, 1 right,
 * 2 up, 3 left, 4 down, 5 right-up, 6 left-up, 7 left-down, 8 right-down.
 * D3Q19: 0 rest, 1..6 the axis pairs (+x,-x,+y,-y,+z,-z), then the twelve
 * edge velocities as opposite pairs.  Textbook weights.                 */

static void set_lattice(kor_t *o, int Q)
{
    static const int c9[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                                 {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    static const int c19[19][3] = {
        {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
        {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
        {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
        {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    o->Q = Q;
    for (int i = 0; i < Q; i++) {
        int nnz = 0;
        for (int a = 0; a < 3; a++) {
            o->c[i][a] = (Q == 9) ? (a < 2 ? c9[i][a] : 0) : c19[i][a];
            nnz += o->c[i][a] != 0;
        }
        if (Q == 9)
            o->w[i] = nnz == 0 ? 4.0 / 9.0 : (nnz == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
        else
            o->w[i] = nnz == 0 ? 1.0 / 3.0 : (nnz == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    /* opposite direction: the one whose velocity is -c_i */
    for (int i = 0; i < Q; i++)
        for (int k = 0; k < Q; k++)
            if (o->c[k][0] == -o->c[i][0] && o->c[k][1] == -o->c[i][1] &&
                o->c[k][2] == -o->c[i][2])
                o->opp[i] = k;
}

static int dir_of(const kor_t *o, const int v[3])
{
    for (int k = 0; k < o->Q; k++)
        if (o->c[k][0] == v[0] && o->c[k][1] == v[1] && o->c[k][2] == v[2]) return k;
    return -1;
}

/* ------------------------------------------------------------------ */
/* Geometry.  x is periodic (Sec. 4.2, inlet/outlet periodic); y and z are
 * periodic only when asked, otherwise whatever lies outside the box is void.
 * Returns 0 and leaves p unchanged when the position lies outside.       */

static int wrap(const kor_t *o, int p[3])
{
    int n[3] = {o->nx, o->ny, o->nz};
    int per[3] = {1, o->periodic_y, o->periodic_z};
    for (int a = 0; a < 3; a++) {
        if (p[a] < 0 || p[a] >= n[a]) {
            if (!per[a]) return 0;
            p[a] = ((p[a] % n[a]) + n[a]) % n[a];
        }
    }
    return 1;
}

static int cell_type(const kor_t *o, const int p_in[3])
{
    int p[3] = {p_in[0], p_in[1], p_in[2]};
    if (!wrap(o, p)) return T_VOID;
    return o->cs_type[p[1] + (long)o->ny * p[2]];
}

static int species_type(int s) { return s == SW ? T_FLUID : T_SOLID; }

static int carries(const kor_t *o, int s, const int p[3])
{
    return cell_type(o, p) == species_type(s);
}

static long cell_index(const kor_t *o, const int p_in[3])
{
    int p[3] = {p_in[0], p_in[1], p_in[2]};
    wrap(o, p);
    return p[0] + (long)o->nx * (p[1] + (long)o->ny * p[2]);
}

/*
 * Source of the streamed population i at cell X of species s (pull form).
 *
 * Sec. 4.2 asks for free-slip at the liquid/solid interface for all three
 * species and for no-slip bounce-back at the outer solid boundaries.  The
 * free-slip rule is applied per link, so that staircase walls are handled:
 *   - the upstream cell X - c_i carries s: plain streaming;
 *   - otherwise A = the axes a with c_ia != 0 whose one-axis neighbour
 *     X - c_ia e_a does not carry s.  The link bounces back (population
 *     opp(i) of X itself) when A is empty (a convex edge), when any blocked
 *     cell is void (outer boundary), or when the interface option is
 *     bounce-back (the Sec. 4.2 alternative for electrons and phonons, and
 *     what the printed Eqs. 19-24 do when read as pairs of opposite
 *     velocities);
 *   - otherwise specular reflection: the components in A are reversed and
 *     the population is pulled from X shifted back along the other axes.
 */
static void stream_source(const kor_t *o, int s, const int X[3], int i, int src[3],
                          int *si)
{
    int up[3] = {X[0] - o->c[i][0], X[1] - o->c[i][1], X[2] - o->c[i][2]};
    if (carries(o, s, up)) {
        memcpy(src, up, sizeof up);
        *si = i;
        return;
    }
    int A[3] = {0, 0, 0}, nA = 0, hits_void = cell_type(o, up) == T_VOID;
    for (int a = 0; a < 3; a++) {
        if (o->c[i][a] == 0) continue;
        int p[3] = {X[0], X[1], X[2]};
        p[a] -= o->c[i][a];
        if (!carries(o, s, p)) {
            A[a] = 1;
            nA++;
            if (cell_type(o, p) == T_VOID) hits_void = 1;
        }
    }
    if (o->iface_bounceback || nA == 0 || hits_void) {
        memcpy(src, X, 3 * sizeof(int));
        *si = o->opp[i];
        return;
    }
    int v[3];
    for (int a = 0; a < 3; a++) {
        v[a] = A[a] ? -o->c[i][a] : o->c[i][a];
        src[a] = A[a] ? X[a] : X[a] - o->c[i][a];
    }
    *si = dir_of(o, v);
}

/* ------------------------------------------------------------------ */
/* Lifetime                                                             */

static void free_stream_cache(kor_t *o)
{
    for (int s = 0; s < 3; s++) {
        free(o->sdx[s]);
        free(o->sy[s]);
        free(o->sz[s]);
        free(o->sdir[s]);
        o->sdx[s] = o->sy[s] = o->sz[s] = o->sdir[s] = NULL;
    }
}

static void build_stream_cache(kor_t *o)
{
    free_stream_cache(o);
    long ncs = (long)o->ny * o->nz;
    for (int s = 0; s < 3; s++) {
        o->sdx[s] = (int *)malloc(sizeof(int) * o->Q * ncs);
        o->sy[s] = (int *)malloc(sizeof(int) * o->Q * ncs);
        o->sz[s] = (int *)malloc(sizeof(int) * o->Q * ncs);
        o->sdir[s] = (int *)malloc(sizeof(int) * o->Q * ncs);
        for (int z = 0; z < o->nz; z++)
            for (int y = 0; y < o->ny; y++) {
                /* x = 1 keeps x - 1 inside the box; any x gives the same rule */
                int X[3] = {o->nx > 1 ? 1 : 0, y, z};
                long q = y + (long)o->ny * z;
                for (int i = 0; i < o->Q; i++) {
                    long k = i * ncs + q;
                    if (!carries(o, s, X)) {
                        o->sdir[s][k] = -1;
                        continue;
                    }
                    int src[3], si;
                    stream_source(o, s, X, i, src, &si);
                    wrap(o, src);
                    o->sdx[s][k] = (o->nx > 1) ? src[0] - X[0] : 0;
                    o->sy[s][k] = src[1];
                    o->sz[s][k] = src[2];
                    o->sdir[s][k] = si;
                }
            }
    }
}

kor_t *kor_create(int Q, int nx, int ny, int nz, int periodic_y, int periodic_z,
                  const unsigned char *cs_type)
{
    if ((Q != 9 && Q != 19) || nx < 1 || ny < 1 || nz < 1) return NULL;
    if (Q == 9 && nz != 1) return NULL;
    kor_t *o = (kor_t *)calloc(1, sizeof(kor_t));
    set_lattice(o, Q);
    o->nx = nx;
    o->ny = ny;
    o->nz = nz;
    o->periodic_y = periodic_y;
    o->periodic_z = periodic_z;
    o->ncell = (long)nx * ny * nz;
    o->cs_type = (unsigned char *)malloc((size_t)ny * nz);
    memcpy(o->cs_type, cs_type, (size_t)ny * nz);
    for (int s = 0; s < 3; s++) {
        o->gs[s] = (double *)calloc((size_t)Q * o->ncell, sizeof(double));
        o->g[s] = (double *)calloc((size_t)Q * o->ncell, sizeof(double));
        o->U[s] = (double *)calloc((size_t)3 * o->ncell, sizeof(double));
        o->U2[s] = (double *)calloc((size_t)3 * o->ncell, sizeof(double));
        o->u[s] = (double *)calloc((size_t)3 * o->ncell, sizeof(double));
        o->F[s] = (double *)calloc((size_t)3 * o->ncell, sizeof(double));
        o->drho[s] = (double *)calloc((size_t)o->ncell, sizeof(double));
    }
    o->rho0 = 1.0;
    for (int s = 0; s < 3; s++) o->tau[s] = 1.0;
    o->iface_bounceback = 0;
    build_stream_cache(o);
    return o;
}

void kor_destroy(kor_t *o)
{
    if (!o) return;
    for (int s = 0; s < 3; s++) {
        free(o->gs[s]);
        free(o->g[s]);
        free(o->U[s]);
        free(o->U2[s]);
        free(o->u[s]);
        free(o->F[s]);
        free(o->drho[s]);
    }
    free_stream_cache(o);
    free(o->cs_type);
    free(o);
}

void kor_set_params(kor_t *o, double tau_w, double tau_e, double tau_p, double rho0,
                    double Gx, double Gy, double Gz, int iface_bounceback)
{
    o->tau[SW] = tau_w;
    o->tau[SE] = tau_e;
    o->tau[SP] = tau_p;
    o->rho0 = rho0;
    o->G[0] = Gx;
    o->G[1] = Gy;
    o->G[2] = Gz;
    if (o->iface_bounceback != iface_bounceback) {
        o->iface_bounceback = iface_bounceback;
        build_stream_cache(o);
    }
}

void kor_set_couplings(kor_t *o, double g_we, double g_wp, double g_ep, double g_ec,
                       double g_pc)
{
    o->g_we = g_we;
    o->g_wp = g_wp;
    o->g_ep = g_ep;
    o->g_ec = g_ec;
    o->g_pc = g_pc;
}

/* ------------------------------------------------------------------ */
/* Thermal fluctuations (Eq. 6: the classical fluctuation-dissipation
 * relation of the fluctuating momentum flux; Eq. 17: its lattice source, a
 * random stress projected on w_i (c_ia c_ib - cs^2 delta_ab)), read as the
 * standard fluctuating lattice Boltzmann method: every non-conserved moment
 * of the post-collision water populations receives Gaussian noise of the
 * variance that the relaxation removes, so that each mode m_k keeps
 * <m_k^2> = mu b_k with mu = rho0 kT / cs^2.  With one relaxation rate for
 * all non-conserved moments (BGK) this is weighted Gaussian noise with its
 * mass and momentum projected out:
 *   a_i = sqrt(w_i) z_i,  z_i ~ N(0, 1) independent,
 *   xi_i = A (a_i - w_i sum_j a_j - 3 w_i c_i . sum_j c_j a_j),
 *   A = sqrt(mu (1 - (1 - omega)^2)) = sqrt(3 rho0 kT omega (2 - omega)),
 * whose stress part is the source of Eq. 17.  Electrons and phonons are not
 * thermalised.
 *
 * Random numbers: the Philox-4x32-10 counter-based generator of Salmon,
 * Moraes, Dror and Shaw (SC 2011), from its definition: ten rounds, each
 * multiplying counter words 0 and 2 by M0 and M1 into 64-bit products and
 * recombining (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), the key bumped by the
 * Weyl constants W0, W1 between rounds.  Counter (cell, step mod 2^32,
 * step / 2^32, k) for k = 0, 1, ...; key = the 64-bit seed.  Each output
 * word r gives u = (r + 1/2) 2^-32, and pairs (u1, u2) give two normals by
 * Box-Muller: sqrt(-2 ln u1) (cos, sin)(2 pi u2).                         */

static void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * c[0], p1 = (uint64_t)M1 * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    memcpy(out, c, sizeof c);
}

/* Q standard normals of one cell and step. */
static void cell_normals(const kor_t *o, long cell, long step, double *z)
{
    const double two32 = 4294967296.0;
    const double pi = 3.14159265358979323846;
    int n = 0;
    for (uint32_t k = 0; n < o->Q; k++) {
        uint32_t ctr[4] = {(uint32_t)cell, (uint32_t)((uint64_t)step & 0xffffffffu),
                           (uint32_t)((uint64_t)step >> 32), k};
        uint32_t r[4];
        philox4x32_10(ctr, o->key, r);
        for (int h = 0; h < 4 && n < o->Q; h += 2) {
            double u1 = ((double)r[h] + 0.5) / two32, u2 = ((double)r[h + 1] + 0.5) / two32;
            double R = sqrt(-2.0 * log(u1));
            z[n++] = R * cos(2.0 * pi * u2);
            if (n < o->Q) z[n++] = R * sin(2.0 * pi * u2);
        }
    }
}

/* Test hook: the four Philox-4x32-10 output words for a counter and key. */
void kor_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out) { philox4x32_10(ctr, key, out); }

/* 7. Thermal noise on the post-collision water populations (see above). */
static void thermal_noise(kor_t *o)
{
    const long N = o->ncell;
    const double om = 1.0 / o->tau[SW];
    const double A = sqrt(3.0 * o->rho0 * o->kT * om * (2.0 - om));
    for (int z = 0; z < o->nz; z++)
        for (int y = 0; y < o->ny; y++)
            for (int x = 0; x < o->nx; x++) {
                int X[3] = {x, y, z};
                if (!carries(o, SW, X)) continue;
                long k = cell_index(o, X);
                double zz[19], a[19], S0 = 0.0, S1[3] = {0.0, 0.0, 0.0};
                cell_normals(o, k, o->step, zz);
                for (int i = 0; i < o->Q; i++) {
                    a[i] = sqrt(o->w[i]) * zz[i];
                    S0 += a[i];
                    for (int d = 0; d < 3; d++) S1[d] += o->c[i][d] * a[i];
                }
                for (int i = 0; i < o->Q; i++) {
                    const int *c = o->c[i];
                    double cS = c[0] * S1[0] + c[1] * S1[1] + c[2] * S1[2];
                    o->gs[SW][i * N + k] += A * (a[i] - o->w[i] * S0 - 3.0 * o->w[i] * cS);
                }
            }
}

void kor_set_fluctuations(kor_t *o, double kT, uint64_t seed)
{
    o->kT = kT;
    o->key[0] = (uint32_t)(seed & 0xffffffffu);
    o->key[1] = (uint32_t)(seed >> 32);
}

/* Second-order polynomial equilibrium in deviation form (Sec. 4: second-order
 * expansion of the local equilibrium in the flow field), rho = rho0 + drho. */
static double geq(const kor_t *o, int i, double drho, const double u[3])
{
    double rho = o->rho0 + drho;
    double cu = o->c[i][0] * u[0] + o->c[i][1] * u[1] + o->c[i][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return o->w[i] * (drho + rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
}

/*
 * Phonons as linear waves (Sec. 3.4): their density obeys the damped wave
 * equation  d_tt n_p - cs^2 d_xx n_p = -gamma_p d_t n_p,  with
 * gamma_p = gamma_pC + gamma_pe (1 - u_e/u_p) the sum of the friction rates.
 * A population set relaxing to an equilibrium that is linear in the
 * momentum,
 *   g^eq_i = w_i [drho + 3 c_i . (rho u)],
 * has the moments drho, rho u and cs^2 drho I (no convective flux rho u u),
 * so continuity d_t n + div j = 0 and momentum d_t j = -cs^2 grad n + F
 * (plus the BGK viscous term) combine into that wave equation once the
 * friction force F of the phonons is inserted.  The forcing term carries only
 * its first moment, (1 - omega/2) w_i 3 c_i . F (the second-moment terms of
 * the Guo source balance the u u part of the second-order equilibrium, which
 * the linear one lacks).
 */
static int wave_species(const kor_t *o, int s) { return s == SP && o->phonon_wave; }

static double geq_species(const kor_t *o, int s, int i, double drho, const double u[3])
{
    if (!wave_species(o, s)) return geq(o, i, drho, u);
    double rho = o->rho0 + drho;
    double cu = o->c[i][0] * u[0] + o->c[i][1] * u[1] + o->c[i][2] * u[2];
    return o->w[i] * (drho + 3.0 * rho * cu);
}

static double guo_species(const kor_t *o, int s, int i, double om, const double u[3],
                          const double F[3])
{
    const int *c = o->c[i];
    double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
    double cF = c[0] * F[0] + c[1] * F[1] + c[2] * F[2];
    double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    if (wave_species(o, s)) return (1.0 - 0.5 * om) * o->w[i] * 3.0 * cF;
    return (1.0 - 0.5 * om) * o->w[i] * (3.0 * (cF - uF) + 9.0 * cu * cF);
}

void kor_set_phonon_wave(kor_t *o, int on) { o->phonon_wave = on != 0; }

/* Start from the local equilibrium of the given fields (dense boxes, one
 * density deviation and three velocity components per species).  The lagged
 * velocities of "steps -1 and -2" are the initial velocity. */
void kor_init_equilibrium(kor_t *o, const double *drho /* [3][ncell] */,
                          const double *u /* [3][3][ncell] */)
{
    long N = o->ncell;
    for (int s = 0; s < 3; s++) {
        memset(o->gs[s], 0, sizeof(double) * o->Q * N);
        memset(o->U[s], 0, sizeof(double) * 3 * N);
        memset(o->U2[s], 0, sizeof(double) * 3 * N);
        for (int z = 0; z < o->nz; z++)
            for (int y = 0; y < o->ny; y++)
                for (int x = 0; x < o->nx; x++) {
                    int p[3] = {x, y, z};
                    if (!carries(o, s, p)) continue;
                    long k = cell_index(o, p);
                    double dr = drho ? drho[s * N + k] : 0.0;
                    double v[3] = {0, 0, 0};
                    for (int a = 0; a < 3 && u; a++) v[a] = u[(s * 3 + a) * N + k];
                    for (int i = 0; i < o->Q; i++) o->gs[s][i * N + k] = geq_species(o, s, i, dr, v);
                    for (int a = 0; a < 3; a++) o->U[s][a * N + k] = v[a];
                    for (int a = 0; a < 3; a++) o->U2[s][a * N + k] = v[a];
                }
    }
    o->step = 0;
}

/* ------------------------------------------------------------------ */
/* Steps 1-4 on the current state: fills g, drho, u, F.                  */

/*
 * Velocity a species shows its interface partners at step n: the mean of its
 * own velocities of steps n-1 and n-2.  The paper's scheme is Markovian
 * (Sec. 4.1) and silent on the time discretisation of the friction; the
 * partner's velocity of the current step is another cell's unfinished work,
 * so the coupling is lagged.  A plain one-step lag turns friction into
 * anti-friction for the period-two (staggered) modes that BGK lattices carry
 * undamped, and grows them; the two-step mean has no period-two component.
 * Both partners use the same two numbers, so the exchange stays exactly
 * antisymmetric (Eq. 27), and a steady state is the same as with no lag.
 */
static double interface_velocity(const kor_t *o, int s, int a, long k)
{
    const long N = o->ncell;
    return 0.5 * (o->U[s][a * N + k] + o->U2[s][a * N + k]);
}

static void stream_and_velocities(kor_t *o)
{
    const long N = o->ncell;
    const int Q = o->Q;

    /* 1. pull-stream */
    for (int s = 0; s < 3; s++)
        for (int z = 0; z < o->nz; z++)
            for (int y = 0; y < o->ny; y++)
                for (int x = 0; x < o->nx; x++) {
                    int X[3] = {x, y, z};
                    if (!carries(o, s, X)) continue;
                    long k = cell_index(o, X);
                    long ncs = (long)o->ny * o->nz, q = y + (long)o->ny * z;
                    for (int i = 0; i < Q; i++) {
                        long e = i * ncs + q;
                        int sx = x + o->sdx[s][e];
                        if (sx < 0) sx += o->nx;
                        if (sx >= o->nx) sx -= o->nx;
                        long ks = sx + (long)o->nx * (o->sy[s][e] + (long)o->ny * o->sz[s][e]);
                        o->g[s][i * N + k] = o->gs[s][o->sdir[s][e] * N + ks];
                    }
                }

    static const int face[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0},
                                   {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};

    for (int z = 0; z < o->nz; z++)
        for (int y = 0; y < o->ny; y++)
            for (int x = 0; x < o->nx; x++) {
                int X[3] = {x, y, z};
                int t = cell_type(o, X);
                if (t == T_VOID) continue;
                long k = cell_index(o, X);

                /* 2. moments of every species living here */
                double dr[3] = {0, 0, 0}, j[3][3] = {{0}};
                for (int s = 0; s < 3; s++) {
                    if (species_type(s) != t) continue;
                    for (int i = 0; i < Q; i++) {
                        double gi = o->g[s][i * N + k];
                        dr[s] += gi;
                        for (int a = 0; a < 3; a++) j[s][a] += o->c[i][a] * gi;
                    }
                }

                /* 3. interface friction over the fluid/solid faces of this cell,
                 *    force density -gamma_kl (Ubar_k - Ubar_l) on species k (Eq. 27). */
                double Fif[3][3] = {{0}};
                for (int f = 0; f < 6; f++) {
                    int nb[3] = {x + face[f][0], y + face[f][1], z + face[f][2]};
                    int tn = cell_type(o, nb);
                    if (t == T_FLUID && tn == T_SOLID) {
                        long kn = cell_index(o, nb);
                        for (int a = 0; a < 3; a++) {
                            double uw = interface_velocity(o, SW, a, k);
                            Fif[SW][a] -= o->g_we * (uw - interface_velocity(o, SE, a, kn));
                            Fif[SW][a] -= o->g_wp * (uw - interface_velocity(o, SP, a, kn));
                        }
                    } else if (t == T_SOLID && tn == T_FLUID) {
                        long kn = cell_index(o, nb);
                        for (int a = 0; a < 3; a++) {
                            double uw = interface_velocity(o, SW, a, kn);
                            Fif[SE][a] += o->g_we * (uw - interface_velocity(o, SE, a, k));
                            Fif[SP][a] += o->g_wp * (uw - interface_velocity(o, SP, a, k));
                        }
                    }
                }

                /* 4. velocities and total forces */
                if (t == T_FLUID) {
                    double rho = o->rho0 + dr[SW];
                    o->drho[SW][k] = dr[SW];
                    for (int a = 0; a < 3; a++) {
                        double Fa = o->G[a] + Fif[SW][a];
                        o->F[SW][a * N + k] = Fa;
                        o->u[SW][a * N + k] = (j[SW][a] + 0.5 * Fa) / rho;
                    }
                } else {
                    double ra = o->rho0 + dr[SE], rb = o->rho0 + dr[SP];
                    double kk = 0.5 * o->g_ep, se = 0.5 * o->g_ec, sp = 0.5 * o->g_pc;
                    double D = (ra + kk + se) * (rb + kk + sp) - kk * kk;
                    o->drho[SE][k] = dr[SE];
                    o->drho[SP][k] = dr[SP];
                    for (int a = 0; a < 3; a++) {
                        double Je = j[SE][a] + 0.5 * Fif[SE][a];
                        double Jp = j[SP][a] + 0.5 * Fif[SP][a];
                        double ue = ((rb + kk + sp) * Je + kk * Jp) / D;
                        double up = ((ra + kk + se) * Jp + kk * Je) / D;
                        o->u[SE][a * N + k] = ue;
                        o->u[SP][a * N + k] = up;
                        o->F[SE][a * N + k] =
                            Fif[SE][a] - o->g_ep * (ue - up) - o->g_ec * ue;
                        o->F[SP][a * N + k] =
                            Fif[SP][a] + o->g_ep * (ue - up) - o->g_pc * up;
                    }
                }
            }
}

/* 6. BGK collision with Guo forcing:
 *    g*_i = g_i + omega (g^eq_i - g_i) + (1 - omega/2) w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F
 *    (phonons of the wave variant: the linear equilibrium and source above) */
static void collide(kor_t *o)
{
    const long N = o->ncell;
    for (int s = 0; s < 3; s++) {
        double om = 1.0 / o->tau[s];
        for (int z = 0; z < o->nz; z++)
            for (int y = 0; y < o->ny; y++)
                for (int x = 0; x < o->nx; x++) {
                    int X[3] = {x, y, z};
                    if (!carries(o, s, X)) continue;
                    long k = cell_index(o, X);
                    double v[3], Fv[3];
                    for (int a = 0; a < 3; a++) {
                        v[a] = o->u[s][a * N + k];
                        Fv[a] = o->F[s][a * N + k];
                    }
                    double dr = o->drho[s][k];
                    for (int i = 0; i < o->Q; i++) {
                        double eq = geq_species(o, s, i, dr, v);
                        double Fi = guo_species(o, s, i, om, v, Fv);
                        double gi = o->g[s][i * N + k];
                        o->gs[s][i * N + k] = gi + om * (eq - gi) + Fi;
                    }
                }
    }
}

void kor_step(kor_t *o, long nsteps)
{
    for (long n = 0; n < nsteps; n++) {
        stream_and_velocities(o);
        /* 5. the velocities of this step are the lagged ones of the next */
        for (int s = 0; s < 3; s++) {
            memcpy(o->U2[s], o->U[s], sizeof(double) * 3 * o->ncell);
            memcpy(o->U[s], o->u[s], sizeof(double) * 3 * o->ncell);
        }
        collide(o);
        if (o->kT > 0.0) thermal_noise(o);
        o->step++;
    }
}

/*
 * Observation at the current step n (after n completed steps): steps 1-4 on
 * the current state, without collision.  Writes the density deviation,
 * velocity and force fields of all species (dense, zero off-species) and the
 * previous-step velocity U.  The state is unchanged.
 */
void kor_observe(kor_t *o, double *drho /* [3][ncell] */, double *u /* [3][3][ncell] */,
                 double *F /* [3][3][ncell] */, double *uprev /* [3][3][ncell] */)
{
    const long N = o->ncell;
    for (int s = 0; s < 3; s++) {
        memset(o->drho[s], 0, sizeof(double) * N);
        memset(o->u[s], 0, sizeof(double) * 3 * N);
        memset(o->F[s], 0, sizeof(double) * 3 * N);
    }
    stream_and_velocities(o);
    for (int s = 0; s < 3; s++) {
        if (drho) memcpy(drho + s * N, o->drho[s], sizeof(double) * N);
        if (u) memcpy(u + s * 3 * N, o->u[s], sizeof(double) * 3 * N);
        if (F) memcpy(F + s * 3 * N, o->F[s], sizeof(double) * 3 * N);
        if (uprev) memcpy(uprev + s * 3 * N, o->U[s], sizeof(double) * 3 * N);
    }
}

long kor_get_step(const kor_t *o) { return o->step; }

/* State access: post-collision deviations [3][Q][ncell] and the lagged
 * velocities U = u(n-1), U2 = u(n-2), each [3][3][ncell]. */
void kor_get_state(const kor_t *o, double *gs, double *U, double *U2)
{
    const long N = o->ncell;
    for (int s = 0; s < 3; s++) {
        if (gs) memcpy(gs + (long)s * o->Q * N, o->gs[s], sizeof(double) * o->Q * N);
        if (U) memcpy(U + (long)s * 3 * N, o->U[s], sizeof(double) * 3 * N);
        if (U2) memcpy(U2 + (long)s * 3 * N, o->U2[s], sizeof(double) * 3 * N);
    }
}

void kor_set_state(kor_t *o, const double *gs, const double *U, const double *U2, long step)
{
    const long N = o->ncell;
    for (int s = 0; s < 3; s++) {
        memcpy(o->gs[s], gs + (long)s * o->Q * N, sizeof(double) * o->Q * N);
        memcpy(o->U[s], U + (long)s * 3 * N, sizeof(double) * 3 * N);
        memcpy(o->U2[s], U2 + (long)s * 3 * N, sizeof(double) * 3 * N);
    }
    o->step = step;
}

/* Streaming source table of one species (for tests of the boundary rule):
 * for every cell and direction, the source cell index and direction, or -1
 * for cells that do not carry the species. */
void kor_stream_table(const kor_t *o, int s, long *src_cell /* [Q][ncell] */,
                      int *src_dir /* [Q][ncell] */)
{
    const long N = o->ncell;
    for (int z = 0; z < o->nz; z++)
        for (int y = 0; y < o->ny; y++)
            for (int x = 0; x < o->nx; x++) {
                int X[3] = {x, y, z};
                long k = cell_index(o, X);
                for (int i = 0; i < o->Q; i++) {
                    if (!carries(o, s, X)) {
                        src_cell[i * N + k] = -1;
                        src_dir[i * N + k] = -1;
                        continue;
                    }
                    int src[3], si;
                    stream_source(o, s, X, i, src, &si);
                    src_cell[i * N + k] = cell_index(o, src);
                    src_dir[i * N + k] = si;
                }
            }
}

/* Lattice tables, for the moment-identity checks. */
void kor_lattice(const kor_t *o, int *c /* [Q][3] */, double *w /* [Q] */, int *opp)
{
    for (int i = 0; i < o->Q; i++) {
        for (int a = 0; a < 3; a++) c[3 * i + a] = o->c[i][a];
        w[i] = o->w[i];
        opp[i] = o->opp[i];
    }
}

/* Equilibrium and Guo source of one direction, exposed for the identity pins. */
double kor_geq(const kor_t *o, int i, double drho, double ux, double uy, double uz)
{
    double u[3] = {ux, uy, uz};
    return geq(o, i, drho, u);
}

/* The same for one species (the phonons differ under the wave variant). */
double kor_geq_species(const kor_t *o, int s, int i, double drho, double ux, double uy, double uz)
{
    double u[3] = {ux, uy, uz};
    return geq_species(o, s, i, drho, u);
}

double kor_guo_species(const kor_t *o, int s, int i, double omega, double ux, double uy, double uz,
                       double Fx, double Fy, double Fz)
{
    double u[3] = {ux, uy, uz}, F[3] = {Fx, Fy, Fz};
    return guo_species(o, s, i, omega, u, F);
}

double kor_guo(const kor_t *o, int i, double omega, double ux, double uy, double uz,
               double Fx, double Fy, double Fz)
{
    const int *c = o->c[i];
    double cu = c[0] * ux + c[1] * uy + c[2] * uz;
    double cF = c[0] * Fx + c[1] * Fy + c[2] * Fz;
    double uF = ux * Fx + uy * Fy + uz * Fz;
    return (1.0 - 0.5 * omega) * o->w[i] * (3.0 * (cF - uF) + 9.0 * cu * cF);
}
