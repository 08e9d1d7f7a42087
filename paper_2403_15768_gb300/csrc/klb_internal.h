// Internal declarations of the KLB library: host geometry tables, device
// memory plan and kernel launchers.  Not part of the public ABI (include/klb.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "klb.h"

namespace klb {

constexpr int kMaxFaces = 4;   // fluid/solid faces of one cross-section cell (+-y, +-z)
constexpr int kBlockX = 128;   // threads per block along x (one x per thread)
// Rows are padded to a multiple of kRowAlign elements.  RowInfo::src counts
// in these units, so a 32-bit entry reaches 2^31 * 32 elements of a class
// buffer; offsets within one direction plane (row * nxp + x) stay 32-bit.
constexpr int kRowAlign = 32;

// Row classes: a row is one cross-section cell together with all its x.
// Water lives on fluid rows; electrons and phonons share the solid rows.
enum RowClass { kFluid = 0, kSolid = 1 };

// Per-row table, read once per block (all threads of a block share a row).
struct RowInfo {
    int32_t src[19];            // (dir' * n_rows + row') * nxp / kRowAlign: first element,
                                // in kRowAlign units, of the row direction i is pulled from
    uint32_t xm;                // bit i: pull direction i from x - 1
    uint32_t xp;                // bit i: pull direction i from x + 1
    int32_t slot;               // interface slot of this row, -1 if none
    int32_t nface;              // number of fluid/solid faces
    int32_t partner[kMaxFaces]; // interface slots of the rows across those faces
    float d2;                   // fluid rows: squared distance to centre plane / axis
    int32_t flags;              // bit 0 in the slip fit, bit 1 wall row (fluid rows);
                                // bit 2: some direction with c_x != 0 bounces back
    int32_t cs;                 // cross-section cell y + ny z (cell x + nx cs of the box)
    int32_t pad[2];
};
static_assert(sizeof(RowInfo) == 128, "RowInfo is one 128-byte line");

enum RowFlags { kFitRow = 1, kWallRow = 2, kXBounce = 4 };

// Indices of the FP64 partial sums reduced by the observation kernel.
enum SumIndex {
    kSumUxFluid = 0,   // sum of u_x over fluid cells
    kSumFitN,          // slip fit: count, sum d^2, sum d^4, sum u, sum u d^2
    kSumFitD2,
    kSumFitD4,
    kSumFitU,
    kSumFitUD2,
    kSumWallN,         // wall-row count and sum u_x
    kSumWallU,
    kSumUxE,           // electron / phonon sum u_x
    kSumUxP,
    kSumMomW,          // sum rho u_x per species
    kSumMomE,
    kSumMomP,
    kSumMassW,         // sum (rho - rho0) per species
    kSumMassE,
    kSumMassP,
    kSumNonfinite,     // count of non-finite rho/u values
    kSumResidual,      // max |u_x(n) - u_x(n-1)| (a max, not a sum)
    kSumClipped,       // 16-bit storage: species-cells with a saturated population
    kNumSums
};

// Host geometry of one lattice (built from the description only).
struct Geometry {
    int Q = 0, nx = 0, ny = 0, nz = 0, nxp = 0;
    int periodic_y = 0, periodic_z = 0;
    std::vector<uint8_t> cs_type;          // ny*nz, index y + ny*z
    std::vector<int> rows[2];              // cross-section index of each row
    std::vector<int> row_of_cs[2];         // row of a cross-section cell, -1 if none
    std::vector<RowInfo> info[2];
    std::vector<int> slot_row[2];          // row of each interface slot
    int max_faces[2] = {0, 0};
    double d_wall = 0.0;
    bool has_fit = false;
};

// Builds the geometry and its streaming / interface tables.  Returns false
// with a message on an invalid description.
bool build_geometry(const klb_desc &d, Geometry &g, std::string &err);

// Offsets (bytes from the caller's buffer) of every device region.
struct MemoryPlan {
    size_t pop[2][3];      // [buffer][species]
    size_t pop_bytes[3];
    size_t U[3][2];        // [time slot][row class]
    size_t U_bytes[2];
    size_t rows[2];
    size_t partials, sums, field;
    size_t field_bytes;
    size_t ref_enc[2][3], ref_dec[2][3];  // [generation][species], reduced storage only
    size_t ref_bytes[3];
    size_t acc, acc_bytes;
    size_t bounds;         // error word of debug builds (KLB_BOUNDS)
    size_t total;
    int nblocks_w, nblocks_s, nchunk, bx;  // one cell per thread (observe, field, init)
    int sbx, snblocks;                     // step kernel: threads per block, blocks
};
MemoryPlan plan_memory(const Geometry &g, int storage);

// Reduced-precision storage: floats per row in the reference tables (Q
// used, padded to a multiple of four), steps between reference refreshes,
// and the power-of-two scale of FP16 differences (keeps them out of the
// subnormal range).
constexpr int kRefStride = 20;
constexpr int kRefEvery = 32;
constexpr float kFp16Scale = 1048576.0f;  // 2^20

// Cells per thread of the step kernel: FP64 one; FP32 arithmetic two
// adjacent x (packed f32x2).  Per row class, so that the classes may differ.
inline int step_cells(int storage, bool water)
{
    (void)water;
    return storage == KLB_FP64 ? 1 : 2;
}

// Step-kernel x chunks per row of the given class for blocks of sbx threads.
inline int step_chunks(int nx, int sbx, int storage, bool water)
{
    const int xb = sbx * step_cells(storage, water);
    return (nx + xb - 1) / xb;
}

inline bool reduced_storage(int storage) { return storage == KLB_FP16_DEV || storage == KLB_BF16_DEV; }
inline size_t storage_bytes(int storage)
{
    return storage == KLB_FP64 ? 8 : (storage == KLB_FP32 ? 4 : 2);
}

// Kernel arguments.  T is the arithmetic type (float or double); the
// populations are stored as T, or as FP16/BF16 against per-row references.
template <typename T>
struct alignas(16) StepArgs {
    const void *in[3];     // current state, per species
    void *out[3];          // next state (step and init modes)
    const void *in_prev[3];  // previous state (observe mode, residual)
    const RowInfo *rows[2];
    const T *U1[2], *U2[2], *U3[2];  // lagged velocities u(n-1), u(n-2), u(n-3)
    T *U0[2];                        // u(n) written here (step mode)
    int nx, nxp, nchunk, nbw;        // nchunk = x chunks of blockDim.x per row; nbw = water blocks
    int snchunk_w, snchunk_s, snbw;  // the same for the step kernel, per row class
    int nch32, nseg_w;               // 32-wide x segments per row; water segments
    int n_rows[2], n_slots[2];
    T rho0, om[3], G[3];
    T g_we, g_wp, g_ep, g_ec, g_pc;
    T q_p;                 // phonons: 1 second-order equilibrium, 0 linear (damped waves, Sec. 3.4)
    double *partials;      // observe mode: [block][kNumSums]
    int residual_valid;
    T *field;              // field / init mode: per species [4][n_rows][nxp]
    // reduced-precision storage only (null otherwise)
    const float *dec_in[3], *dec_prev[3];  // references of pulled populations
    const float *enc_out[3];               // references of stored populations
    float scale, inv_scale;
    float *acc;            // x-sums of g* per 32-wide segment [segment][2Q]
    // thermal fluctuations of the water (step with noise only)
    T noise_amp;           // sqrt(3 rho0 kT omega (2 - omega))
    uint32_t key[2];       // generator key (seed)
    uint32_t step_lo, step_hi;  // the step being taken
    // batches: the record is of a period's phase, replayed; the step taken is
    // step_lo + *step_reps * step_period (low 32 bits), step_reps counting the
    // periods completed since the tables were built (null for one lattice)
    const uint32_t *step_reps;
    int step_period;
    unsigned *bounds_err;  // debug builds: first out-of-range index site
};

enum Mode {
    kModeStep = 0,
    kModeObserve = 1,
    kModeField = 2,
    kModeStepAcc = 3,  // step that also writes the x-sums for a refresh
    kModeInit = 4,
    kModeInitAcc = 5,  // x-sums of the initial equilibria, nothing stored
    kModeStepNoise = 6 // step with thermal fluctuations of the water
};

// Launchers (return the launch error, if any).
cudaError_t launch(int Q, int storage, const void *args, int mode, int nblocks, int bx,
                   cudaStream_t s);
// Reference refresh from args.acc into the tables enc[s], dec[s].
cudaError_t launch_ref(int Q, int storage, const void *args, float *const enc[3],
                       float *const dec[3], cudaStream_t s);
cudaError_t launch_finalize(const double *partials, int nblocks, double *sums, cudaStream_t s);
// One more period completed by a batch (StepArgs::step_reps).
cudaError_t launch_count_period(uint32_t *reps, cudaStream_t s);
// One step of many lattices in one launch: table[l] holds the arguments of
// lattice l, prefix[l] its first block (prefix[n] = total blocks).
cudaError_t launch_batch(int Q, int storage, const void *table, const int *prefix, int n,
                         int nblocks, int bx, bool acc, cudaStream_t s);

// Device bytes of the argument tables of a batch of n lattices with this
// storage (the layout klb_batch_create uses).
size_t batch_table_bytes(int storage, int n);

// Observation pass of a lattice enqueued on its stream, its kNumSums sums copied
// to host_sums (pinned host memory; valid after the stream synchronises),
// and the observables computed from them (klb_observables in two halves).
cudaError_t observe_enqueue(klb_lattice *L, double *host_sums);
klb_status observe_finish(klb_lattice *L, const double *host_sums, klb_obs *out);

// Static scratch of klb_observables_static (klb_static.cu): device addresses
// of its partial-sum rows and final sums on the current device.
cudaError_t static_scratch(double **partials, double **sums, size_t *max_blocks);

}  // namespace klb
