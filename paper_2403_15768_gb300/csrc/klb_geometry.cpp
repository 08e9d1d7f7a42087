// Host-side geometry of a KLB lattice: the cross-section type map of the
// channel (Sec. 2: water in a nanochannel between solid walls), the compact
// row numbering of each species class, the pull-streaming source of every
// (row, direction) with the boundary rules of Sec. 4.2, and the fluid/solid
// interface faces that carry the friction of Eq. 27.
//
// The channel is x-invariant and periodic in x, so everything here is a
// property of the (y, z) cross-section; the kernels apply it to every x.

#include <algorithm>
#include <cmath>
#include <cstring>

#include "klb_internal.h"

namespace klb {

namespace {

enum { kVoid = 0, kFluidCell = 1, kSolidCell = 2 };

struct Velocities {
    int Q;
    int c[19][3];
    int opp[19];
};

Velocities make_velocities(int Q)
{
    // D2Q9 in the numbering of Sec. 4.2; D3Q19 as documented in klb.h.
    static const int v9[9][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
                                 {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
    static const int v19[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                                   {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                   {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                   {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    Velocities v;
    v.Q = Q;
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < 3; ++a) v.c[i][a] = (Q == 9) ? v9[i][a] : v19[i][a];
    for (int i = 0; i < Q; ++i)
        for (int k = 0; k < Q; ++k)
            if (v.c[k][0] == -v.c[i][0] && v.c[k][1] == -v.c[i][1] && v.c[k][2] == -v.c[i][2])
                v.opp[i] = k;
    return v;
}

int find_dir(const Velocities &v, int cx, int cy, int cz)
{
    for (int k = 0; k < v.Q; ++k)
        if (v.c[k][0] == cx && v.c[k][1] == cy && v.c[k][2] == cz) return k;
    return -1;
}

struct CrossSection {
    int ny, nz, per_y, per_z;
    const std::vector<uint8_t> *t;
    // Wraps (y, z) along periodic axes; false if it lies outside the box.
    bool wrap(int &y, int &z) const
    {
        if (y < 0 || y >= ny) {
            if (!per_y) return false;
            y = ((y % ny) + ny) % ny;
        }
        if (z < 0 || z >= nz) {
            if (!per_z) return false;
            z = ((z % nz) + nz) % nz;
        }
        return true;
    }
    int type(int y, int z) const { return wrap(y, z) ? (int)(*t)[y + ny * z] : (int)kVoid; }
    int index(int y, int z) const
    {
        wrap(y, z);
        return y + ny * z;
    }
};

int class_cell_type(int cls) { return cls == kFluid ? kFluidCell : kSolidCell; }

bool finite_all(const double *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

}  // namespace

bool build_geometry(const klb_desc &d, Geometry &g, std::string &err)
{
    if (d.kind != KLB_D2Q9 && d.kind != KLB_D3Q19) return err = "kind must be KLB_D2Q9 or KLB_D3Q19", false;
    if (d.nx < 1 || d.ny < 1 || d.nz < 1) return err = "nx, ny, nz must be >= 1", false;
    if (d.kind == KLB_D2Q9 && d.nz != 1) return err = "D2Q9 needs nz == 1", false;
    if (d.storage != KLB_FP64 && d.storage != KLB_FP32 && !reduced_storage(d.storage))
        return err = "storage must be KLB_FP64, KLB_FP32, KLB_FP16_DEV or KLB_BF16_DEV", false;
    if (d.iface_bc != KLB_IFACE_SPECULAR && d.iface_bc != KLB_IFACE_BOUNCEBACK)
        return err = "iface_bc must be SPECULAR or BOUNCEBACK", false;
    if (d.phonon_eq != KLB_PHONON_FLUID && d.phonon_eq != KLB_PHONON_WAVE)
        return err = "phonon_eq must be KLB_PHONON_FLUID or KLB_PHONON_WAVE", false;
    double taus[3] = {d.tau_w, d.tau_e, d.tau_p};
    if (!finite_all(taus, 3) || !finite_all(&d.rho0, 1) || !finite_all(d.G, 3))
        return err = "non-finite tau, rho0 or G", false;
    for (double t : taus)
        if (!(t > 0.5)) return err = "relaxation times must exceed 1/2", false;
    if (!(d.rho0 > 0)) return err = "rho0 must be positive", false;

    g = Geometry();
    g.Q = d.kind;
    g.nx = d.nx;
    g.ny = d.ny;
    g.nz = d.nz;
    g.nxp = (d.nx + 31) / 32 * 32;
    g.cs_type.assign((size_t)d.ny * d.nz, kVoid);

    // ---- cross-section type map
    if (d.geom == KLB_GEOM_SLAB) {
        if (d.width < 1 || d.shell < 1 || d.width + 2 * d.shell > d.ny)
            return err = "slab needs width >= 1, shell >= 1, width + 2 shell <= ny", false;
        int y0 = (d.ny - d.width) / 2;
        for (int z = 0; z < d.nz; ++z)
            for (int y = 0; y < d.ny; ++y) {
                int t = kVoid;
                if (y >= y0 && y < y0 + d.width)
                    t = kFluidCell;
                else if (y >= y0 - d.shell && y < y0 + d.width + d.shell)
                    t = kSolidCell;
                g.cs_type[y + (size_t)d.ny * z] = (uint8_t)t;
            }
        g.periodic_y = 0;
        g.periodic_z = 1;
    } else if (d.geom == KLB_GEOM_PIPE) {
        if (d.radius < 1 || d.shell < 1) return err = "pipe needs radius >= 1 and shell >= 1", false;
        // r of the cell centre (y + 1/2, z + 1/2) about (ny/2, nz/2), compared
        // exactly in doubled integer coordinates.
        const long rf = 2L * d.radius, rs = 2L * (d.radius + d.shell);
        for (int z = 0; z < d.nz; ++z)
            for (int y = 0; y < d.ny; ++y) {
                long dy = 2L * y + 1 - d.ny, dz = 2L * z + 1 - d.nz;
                long r2 = dy * dy + dz * dz;
                int t = r2 < rf * rf ? kFluidCell : (r2 < rs * rs ? kSolidCell : kVoid);
                g.cs_type[y + (size_t)d.ny * z] = (uint8_t)t;
            }
        g.periodic_y = 0;
        g.periodic_z = 0;
    } else if (d.geom == KLB_GEOM_MASK) {
        if (!d.mask) return err = "MASK geometry needs a mask", false;
        for (size_t k = 0; k < g.cs_type.size(); ++k) {
            if (d.mask[k] > 2) return err = "mask values must be 0, 1 or 2", false;
            g.cs_type[k] = d.mask[k];
        }
        g.periodic_y = d.periodic_y != 0;
        g.periodic_z = d.periodic_z != 0;
    } else {
        return err = "unknown geometry", false;
    }

    CrossSection cs{d.ny, d.nz, g.periodic_y, g.periodic_z, &g.cs_type};
    const Velocities v = make_velocities(g.Q);
    const int ncs = d.ny * d.nz;

    // ---- compact rows per class
    for (int cls = 0; cls < 2; ++cls) {
        g.row_of_cs[cls].assign(ncs, -1);
        for (int k = 0; k < ncs; ++k)
            if (g.cs_type[k] == class_cell_type(cls)) {
                g.row_of_cs[cls][k] = (int)g.rows[cls].size();
                g.rows[cls].push_back(k);
            }
    }
    if (g.rows[kFluid].empty()) return err = "geometry has no fluid cells", false;
    if (g.rows[kSolid].empty()) return err = "geometry has no solid cells", false;
    // Index widths: a cell of the box is a 32-bit number x + nx (y + ny z);
    // offsets within one direction plane (row * nxp + x) and within the
    // interface-velocity buffers are 32-bit; row sources count in kRowAlign
    // units of a class buffer (Q planes).  Larger class buffers than 2^31
    // elements are fine: plane strides are 64-bit in the kernels.
    if ((double)d.nx * d.ny * d.nz >= 4294967296.0)
        return err = "box too large for 32-bit cell indices", false;
    for (int cls = 0; cls < 2; ++cls) {
        const double plane = (double)g.rows[cls].size() * g.nxp;
        if (plane >= 2147483648.0 || (double)g.Q * plane / kRowAlign >= 2147483648.0)
            return err = "lattice too large for 32-bit row offsets", false;
    }

    // ---- interface faces and slots
    const int face_dir[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
    const int nfaces_dirs = (g.Q == 9) ? 2 : 4;
    for (int cls = 0; cls < 2; ++cls) {
        const int other = 1 - cls;
        const size_t nr = g.rows[cls].size();
        g.info[cls].assign(nr, RowInfo());
        for (size_t r = 0; r < nr; ++r) {
            RowInfo &ri = g.info[cls][r];
            std::memset(&ri, 0, sizeof ri);
            ri.slot = -1;
            int k = g.rows[cls][r], y = k % d.ny, z = k / d.ny;
            ri.cs = k;
            for (int f = 0; f < nfaces_dirs; ++f) {
                int yy = y + face_dir[f][0], zz = z + face_dir[f][1];
                if (cs.type(yy, zz) == class_cell_type(other)) {
                    ri.partner[ri.nface++] = cs.index(yy, zz);  // cross-section index for now
                }
            }
            if (ri.nface > 0) {
                ri.slot = (int)g.slot_row[cls].size();
                g.slot_row[cls].push_back((int)r);
            }
            g.max_faces[cls] = std::max(g.max_faces[cls], (int)ri.nface);
        }
    }
    for (int cls = 0; cls < 2; ++cls)
        if ((cls == kFluid ? 3.0 : 6.0) * g.slot_row[cls].size() * g.nxp >= 2147483648.0)
            return err = "lattice too large for 32-bit interface offsets", false;
    // partner cross-section index -> partner slot
    for (int cls = 0; cls < 2; ++cls)
        for (RowInfo &ri : g.info[cls])
            for (int f = 0; f < ri.nface; ++f) {
                int prow = g.row_of_cs[1 - cls][ri.partner[f]];
                ri.partner[f] = g.info[1 - cls][prow].slot;
            }

    // ---- pull-streaming sources (Sec. 4.2).  For a row of class cls and
    // direction i, the upstream cross-section cell (y - c_y, z - c_z):
    //   carries the class            -> plain streaming, x shifted by c_x;
    //   otherwise, with A the blocked transverse axes (c_a != 0 and the
    //   one-axis neighbour does not carry the class):
    //     bounce-back (same cell, opposite direction, no x shift) when the
    //     interface option is bounce-back, when A is empty (convex edge), or
    //     when the upstream cell or a blocked neighbour is void (outer wall);
    //     else free-slip (specular): reverse the blocked components, pull
    //     from the cell shifted back along the unblocked axes.
    for (int cls = 0; cls < 2; ++cls) {
        const int ct = class_cell_type(cls);
        const int nr = (int)g.rows[cls].size();
        for (int r = 0; r < nr; ++r) {
            RowInfo &ri = g.info[cls][r];
            int k = g.rows[cls][r], y = k % d.ny, z = k / d.ny;
            for (int i = 0; i < g.Q; ++i) {
                const int cx = v.c[i][0], cy = v.c[i][1], cz = v.c[i][2];
                int sy = y - cy, sz = z - cz, sdir = i, sx = cx;
                int tu = cs.type(y - cy, z - cz);
                if (tu != ct) {
                    bool Ay = cy != 0 && cs.type(y - cy, z) != ct;
                    bool Az = cz != 0 && cs.type(y, z - cz) != ct;
                    bool hits_void = tu == kVoid || (Ay && cs.type(y - cy, z) == kVoid) ||
                                     (Az && cs.type(y, z - cz) == kVoid);
                    if (d.iface_bc == KLB_IFACE_BOUNCEBACK || (!Ay && !Az) || hits_void) {
                        sy = y;
                        sz = z;
                        sdir = v.opp[i];
                        sx = 0;
                    } else {
                        sy = Ay ? y : y - cy;
                        sz = Az ? z : z - cz;
                        sdir = find_dir(v, cx, Ay ? -cy : cy, Az ? -cz : cz);
                    }
                }
                int srow = g.row_of_cs[cls][cs.index(sy, sz)];
                if (srow < 0 || sdir < 0) return err = "internal: streaming source off the species", false;
                ri.src[i] = (int32_t)(((long)sdir * nr + srow) * (g.nxp / kRowAlign));
                if (sx == 1) ri.xm |= 1u << i;   // source at x - 1
                if (sx == -1) ri.xp |= 1u << i;  // source at x + 1
                if (cx != 0 && sx == 0) ri.flags |= kXBounce;
            }
        }
        // Every population must be pulled exactly once (mass conservation).
        std::vector<uint8_t> used((size_t)g.Q * nr, 0);
        for (int r = 0; r < nr; ++r)
            for (int i = 0; i < g.Q; ++i) {
                long e = g.info[cls][r].src[i] / (g.nxp / kRowAlign);
                if (used[e]++) return err = "boundary rule is not a permutation for this geometry", false;
            }
    }

    // ---- slip-fit and wall-row flags of fluid rows
    int n_fluid = (int)g.rows[kFluid].size();
    if (d.geom == KLB_GEOM_SLAB) {
        g.d_wall = d.width / 2.0;
        g.has_fit = true;
    } else if (d.geom == KLB_GEOM_PIPE) {
        g.d_wall = std::sqrt(n_fluid / M_PI);
        g.has_fit = true;
    }
    for (int r = 0; r < n_fluid; ++r) {
        RowInfo &ri = g.info[kFluid][r];
        int k = g.rows[kFluid][r], y = k % d.ny, z = k / d.ny;
        double dist = 0.0;
        if (d.geom == KLB_GEOM_SLAB) {
            double yc = (d.ny - d.width) / 2 + d.width / 2.0;
            dist = std::fabs(y + 0.5 - yc);
        } else if (d.geom == KLB_GEOM_PIPE) {
            long dy = 2L * y + 1 - d.ny, dz = 2L * z + 1 - d.nz;
            dist = std::sqrt((double)(dy * dy + dz * dz)) / 2.0;
        }
        ri.d2 = (float)(dist * dist);
        if (g.has_fit && (g.d_wall - dist) >= 4.0) ri.flags |= kFitRow;
        if (ri.nface > 0) ri.flags |= kWallRow;
    }
    return true;
}

MemoryPlan plan_memory(const Geometry &g, int storage)
{
    MemoryPlan p;
    const size_t ss = storage_bytes(storage);            // population storage
    const size_t ts = storage == KLB_FP64 ? 8 : 4;       // arithmetic type
    const size_t nr[2] = {g.rows[kFluid].size(), g.rows[kSolid].size()};
    const size_t ns[2] = {g.slot_row[kFluid].size(), g.slot_row[kSolid].size()};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off += (bytes + 255) / 256 * 256;
        return at;
    };
    for (int s = 0; s < 3; ++s) p.pop_bytes[s] = ss * g.Q * nr[s == 0 ? kFluid : kSolid] * g.nxp;
    for (int b = 0; b < 2; ++b)
        for (int s = 0; s < 3; ++s) p.pop[b][s] = take(p.pop_bytes[s]);
    p.U_bytes[kFluid] = ts * 3 * ns[kFluid] * g.nxp;
    p.U_bytes[kSolid] = ts * 6 * ns[kSolid] * g.nxp;
    for (int t = 0; t < 3; ++t)
        for (int c = 0; c < 2; ++c) p.U[t][c] = take(p.U_bytes[c]);
    p.rows[kFluid] = take(sizeof(RowInfo) * nr[kFluid]);
    p.rows[kSolid] = take(sizeof(RowInfo) * nr[kSolid]);
    p.bx = std::min(kBlockX, std::max(32, (g.nx + 31) / 32 * 32));
    p.nchunk = (g.nx + p.bx - 1) / p.bx;
    p.nblocks_w = (int)nr[kFluid] * p.nchunk;
    p.nblocks_s = (int)nr[kSolid] * p.nchunk;
    {
        const int c = step_cells(storage, false);
        const int xt = (g.nx + c - 1) / c;  // threads per solid row
        p.sbx = std::min(kBlockX, std::max(32, (xt + 31) / 32 * 32));
        p.snblocks = (int)nr[kFluid] * step_chunks(g.nx, p.sbx, storage, true) +
                     (int)nr[kSolid] * step_chunks(g.nx, p.sbx, storage, false);
    }
    p.partials = take(sizeof(double) * kNumSums * (size_t)(p.nblocks_w + p.nblocks_s));
    p.sums = take(sizeof(double) * kNumSums);
    p.field_bytes = ts * 4 * (nr[kFluid] + 2 * nr[kSolid]) * g.nxp;
    p.field = take(p.field_bytes);
    for (int s = 0; s < 3; ++s) p.ref_bytes[s] = 0;
    p.acc = p.acc_bytes = 0;
    for (int gen = 0; gen < 2; ++gen)
        for (int s = 0; s < 3; ++s) p.ref_enc[gen][s] = p.ref_dec[gen][s] = 0;
    if (reduced_storage(storage)) {
        for (int s = 0; s < 3; ++s)
            p.ref_bytes[s] = sizeof(float) * kRefStride * nr[s == 0 ? kFluid : kSolid];
        for (int gen = 0; gen < 2; ++gen)
            for (int s = 0; s < 3; ++s) {
                p.ref_enc[gen][s] = take(p.ref_bytes[s]);
                p.ref_dec[gen][s] = take(p.ref_bytes[s]);
            }
        const size_t nseg = (nr[kFluid] + nr[kSolid]) * (size_t)((g.nx + 31) / 32);
        p.acc_bytes = sizeof(float) * 2 * g.Q * nseg;
        p.acc = take(p.acc_bytes);
    }
    p.bounds = take(sizeof(unsigned));
    p.total = off;
    return p;
}

}  // namespace klb
