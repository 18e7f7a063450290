// md_api.cu -- host implementation of the C ABI declared in include/md.h.
//
// The handle carves every device array out of the caller's workspace, keeps
// the per-replica tables there, and drives the kernels on the caller's stream.
// md_step() runs as one CUDA graph:
//
//   integrate(FIRST) -> IF(rebuild){bin, scan, scatter, permute, nbuild}
//     -> WHILE(loop){ step x c -> IF(rebuild){...} -> step x c -> IF ... }
//
// with kUnroll step kernels per loop iteration and a rebuild check after every
// c of them (the check interval).  The last block of each kernel sets the
// conditions on the device (rebuild when the displacement since the last
// build, plus a bound on the motion until the next check, could exceed
// skin/2; loop while steps
// remain), so a whole md_step of n steps is one graph launch with no host
// round trip.  Conditional nodes cost microseconds each on this hardware,
// which is why the loop is unrolled and the check is spaced.  With
// use_graph = 0 the same kernel sequence, with the same check points, is
// launched from the host (the results are bitwise identical).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "md.h"
#include "md_tables.h"
#include "md_common.cuh"
#include "md_corr.cuh"

static_assert(sizeof(md_params) == 192, "md_params layout is part of the ABI");

using mdk::KArgs;
using mdk::KernelSet;

// md_noalloc.cu: message of the calling thread's last failed handle-free call
const char *md_noalloc_message();

namespace {
// A named range on a profiler's host timeline for the duration of one API call
// (NVTX; costs nothing when no tool is attached).
struct ApiRange {
    explicit ApiRange(const char *name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
    ApiRange(const ApiRange &) = delete;
    ApiRange &operator=(const ApiRange &) = delete;
};
}  // namespace

namespace {

constexpr size_t kAlign = 256;
constexpr int kIntBlock = 256, kForceBlock = 128, kScanBlock = 1024;
constexpr int kNbWarpCellsPerSm = 8;                     // warp-per-cell build from this many cells per SM
constexpr int kNbCells = 4, kNbBlock = 32 * kNbCells;   // neighbour build: one warp per cell ...
constexpr int kNbBlockB = 256;                          // ... or one block per cell
constexpr double kCellMargin = 1e-3;   // cell edge exceeds the largest list radius by this
constexpr int kUnroll = 16;            // step kernels per loop iteration of the graph
constexpr int kCheck = 4;              // automatic check interval below kCheckLargeN particles
constexpr int64_t kCheckLargeN = 262144;   // from here a check after every step: the conditional
                                           // node costs little against the step, the earlier
                                           // rebuilds of a long interval cost more

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Everything that follows from the parameters and the replica sizes.
struct Geometry {
    int R = 0;
    int64_t n = 0;
    int K = 0, Kmax = 0, tpp = 8, ppb_f = 32;   // starting list capacity, its cap
    int check = kCheck;                 // MD steps between rebuild checks of the graph
    bool nb_block = false;              // neighbour build with one block (8 warps) per cell
    int nblk_i = 0, nblk_f = 0, ncell = 0;
    bool sweep = false;                 // step kernel: resident blocks sweeping runs of chunks
    int nblk_s = 0, cpb = 1;            // step kernel: blocks launched, chunks per block
    double rl_max = 0.0;
    std::vector<mdk::Rep> rep;
    std::vector<int4> blk_i, blk_f;
    std::vector<int> crank;
    std::vector<int4> cxyz;
};

struct Layout {
    size_t off_ctl, off_rep, off_blk_i, off_blk_f, off_blk_s, off_crank, off_cxyz;
    size_t off_pa, off_pb, off_va, off_vb, off_pa2, off_pb2, off_va2, off_vb2, off_qa, off_qb, off_force;
    size_t off_rref, off_image, off_image2, off_key, off_tmpidx, off_skey;
    size_t off_ccount, off_ccursor, off_cstart, off_nbr, off_nnbr, off_part_f, off_part_i, off_part_e;
    size_t off_ring, off_totals, off_scale, off_st_pos, off_st_vel, off_st_img, off_st_code;
    size_t off_epot, off_epot_step;
    size_t off_st_f, off_st_e, total;
};

int prec_pos_bytes(int prec) { return prec == MD_PREC_FP64 ? 32 : 16; }

// Index of cell (x, y, z) along the Hilbert curve through a 2^b cube: the
// coordinates are transformed in place (Skilling's transposition method,
// "Programming the Hilbert curve", AIP Conf. Proc. 707, 2004), then their bits
// are interleaved, most significant first.
uint32_t hilbert3(uint32_t x, uint32_t y, uint32_t z, int b)
{
    uint32_t X[3] = {x, y, z};
    const uint32_t top = 1u << (b - 1);
    for (uint32_t q = top; q > 1; q >>= 1) {
        const uint32_t low = q - 1;
        for (int i = 0; i < 3; ++i) {
            if (X[i] & q) {
                X[0] ^= low;                          // reflect the lower bits of axis 0
            } else {
                const uint32_t t = (X[0] ^ X[i]) & low;   // exchange them with axis i
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];                                     // Gray code across the axes
    X[2] ^= X[1];
    uint32_t t = 0;
    for (uint32_t q = top; q > 1; q >>= 1)
        if (X[2] & q)
            t ^= q - 1;
    for (int i = 0; i < 3; ++i)
        X[i] ^= t;
    uint32_t h = 0;
    for (int k = b - 1; k >= 0; --k)
        for (int i = 0; i < 3; ++i)
            h = (h << 1) | ((X[i] >> k) & 1u);
    return h;
}

uint32_t spread3(uint32_t v)
{
    uint32_t r = 0;
    for (int b = 0; b < 10; ++b)
        r |= ((v >> b) & 1u) << (3 * b);
    return r;
}

int auto_capacity(const md_params *p, const Geometry &g, const std::vector<double> &box,
                  const std::vector<int64_t> &nrep)
{
    double rho = 0.0;
    for (size_t r = 0; r < box.size(); ++r)
        rho = std::max(rho, (double)nrep[r] / (box[r] * box[r] * box[r]));
    const double nl = 4.18879020478639 * g.rl_max * g.rl_max * g.rl_max * rho;   // 4/3 pi r^3 rho
    int k = (int)std::ceil(1.35 * nl + 24.0);
    k = (k + 31) / 32 * 32;
    (void)p;
    return std::max(k, 32);
}

// Returns MD_OK or MD_E_INVAL with *msg set.
int make_geometry(const md_params *p, int R, const int64_t *nrep, const double *box, Geometry &g,
                  std::string &msg)
{
    if (!p || R < 1 || !nrep || !box) {
        msg = "null argument or n_replicas < 1";
        return MD_E_INVAL;
    }
    if (p->n_species < 1 || p->n_species > 2) { msg = "n_species must be 1 or 2"; return MD_E_INVAL; }
    if (!(p->dt > 0.0) || !std::isfinite(p->dt)) { msg = "dt must be positive"; return MD_E_INVAL; }
    if (!(p->skin >= 0.0)) { msg = "skin must be >= 0"; return MD_E_INVAL; }
    if (p->precision < 0 || p->precision > 2) { msg = "unknown precision mode"; return MD_E_INVAL; }
    if (p->sample_interval < 1) { msg = "sample_interval must be >= 1"; return MD_E_INVAL; }
    const int tpp = p->threads_per_particle;
    if (tpp != 0 && (tpp < 1 || tpp > 32 || (tpp & (tpp - 1)))) {
        msg = "threads_per_particle must be 0 or a power of two in [1, 32]";
        return MD_E_INVAL;
    }
    if (p->step_form < 0 || p->step_form > 2) {
        msg = "step_form must be 0 (automatic), 1 (one block per chunk) or 2 (resident blocks sweep)";
        return MD_E_INVAL;
    }
    if (p->build_form < 0 || p->build_form > 2) {
        msg = "build_form must be 0 (automatic), 1 (warp per cell) or 2 (block per cell)";
        return MD_E_INVAL;
    }
    if (p->neigh_capacity < 0 || p->neigh_capacity_max < 0) {
        msg = "neigh_capacity and neigh_capacity_max must be >= 0";
        return MD_E_INVAL;
    }
    if (p->step_budget < 0) { msg = "step_budget must be >= 0"; return MD_E_INVAL; }
    {
        const int ci = p->check_interval;
        if (ci != 0 && (ci < 1 || ci > kUnroll || (ci & (ci - 1)) || kUnroll % ci)) {
            msg = "check_interval must be 0 (automatic) or 1, 2, 4, 8 or 16";
            return MD_E_INVAL;
        }
    }
    if (!(p->smooth_h >= 0.0) || !std::isfinite(p->smooth_h)) {
        msg = "smooth_h must be finite and >= 0";
        return MD_E_INVAL;
    }
    if (p->reorder < 0 || p->reorder > 2) {
        msg = "reorder must be 0 (x-fastest), 1 (Morton) or 2 (Hilbert)";
        return MD_E_INVAL;
    }
    if (p->smooth_h > 0.0 && tpp > 8) {
        msg = "threads_per_particle above 8 is not available with the smoothed potential";
        return MD_E_INVAL;
    }
    const int ns = p->n_species;
    double rcmax = 0.0;
    for (int a = 0; a < ns; ++a) {
        if (!(p->mass[a] > 0.0)) { msg = "masses must be positive"; return MD_E_INVAL; }
        for (int b = 0; b < ns; ++b) {
            if (p->eps[a][b] != p->eps[b][a] || p->sigma[a][b] != p->sigma[b][a] ||
                p->rcut[a][b] != p->rcut[b][a]) {
                msg = "pair parameters must be symmetric";
                return MD_E_INVAL;
            }
            if (!(p->sigma[a][b] > 0.0) || !(p->rcut[a][b] > 0.0)) {
                msg = "sigma and rcut must be positive";
                return MD_E_INVAL;
            }
            rcmax = std::max(rcmax, p->rcut[a][b]);
        }
    }
    g.R = R;
    g.rl_max = rcmax + p->skin + (double)mdk::kListMargin;
    // lanes per particle: 2 for the FP32 pair loops (4096 warps at KA N=65536 fit one wave at
    // 64 registers), 4 for FP64 (measured on GB300)
    g.tpp = tpp ? tpp : (p->precision == MD_PREC_FP64 ? 4 : 2);
    g.ppb_f = kForceBlock / g.tpp;
    if (p->step_form == 2 && (p->precision == MD_PREC_FP64 || g.tpp > 2)) {
        msg = "step_form 2 needs MIXED or FP32 and 1 or 2 threads per particle";
        return MD_E_INVAL;
    }
    g.n = 0;
    g.rep.assign(R, mdk::Rep{});
    g.blk_i.clear();
    g.blk_f.clear();
    g.crank.clear();
    g.cxyz.clear();
    int cell0 = 0;
    for (int r = 0; r < R; ++r) {
        const double L = box[r];
        if (nrep[r] < 2) { msg = "every replica needs at least 2 particles"; return MD_E_INVAL; }
        if (!(L > 2.0 * g.rl_max)) {
            char b[160];
            snprintf(b, sizeof b, "box %d (L = %g) must exceed twice the largest cutoff plus skin (%g)",
                     r, L, 2.0 * g.rl_max);
            msg = b;
            return MD_E_INVAL;
        }
        if (g.n + nrep[r] > (int64_t)(1 << 30)) { msg = "too many particles"; return MD_E_INVAL; }
        mdk::Rep &q = g.rep[r];
        q.start = (int)g.n;
        q.n = (int)nrep[r];
        int nc = (int)std::floor(L / (g.rl_max + kCellMargin));
        if (nc < 3)
            nc = 1;
        if (nc > 1024)
            nc = 1024;
        q.nc = nc;
        q.cell0 = cell0;
        q.L = L;
        q.invL = 1.0 / L;
        q.cscale = nc / L;
        q.invLf = (float)(1.0 / L);
        q.cscalef = (float)(nc / L);
        q.qunit = (float)(L / 4294967296.0);
        q.qscale = (float)(4294967296.0 / L);
        // anchoring grid: smallest power of two with 2L < 2^24 * grid
        int e = (int)std::ceil(std::log2(2.0 * L)) - 24;
        double grid = std::ldexp(1.0, e);
        while (2.0 * L >= grid * 16777216.0)
            grid *= 2.0;
        q.grid = (float)grid;
        q.inv_grid = (float)(1.0 / grid);
        // grid * 2^32 / L lies in (2^9, 2^10]: times 2^28 it fits 38 bits, and times the
        // anchored high word's grid index (< 2^24) 62 bits
        q.qgrid = (unsigned long long)std::llround(grid * 4294967296.0 / L * 268435456.0);
        if (p->precision == MD_PREC_MIXED) {
            const double lh = std::rint(L / grid) * grid;
            q.Lhi = (float)lh;
            q.Llo = (float)(L - lh);
        } else {
            q.Lhi = (float)L;
            q.Llo = (float)(L - (double)(float)L);
        }
        // integrate-kernel blocks
        q.bi0 = (int)g.blk_i.size();
        for (int s = 0; s < q.n; s += kIntBlock)
            g.blk_i.push_back(make_int4(q.start + s, q.start + std::min(q.n, s + kIntBlock), r, 0));
        q.bi1 = (int)g.blk_i.size();
        q.bf0 = (int)g.blk_f.size();
        for (int s = 0; s < q.n; s += g.ppb_f)
            g.blk_f.push_back(make_int4(q.start + s, q.start + std::min(q.n, s + g.ppb_f), r, 0));
        q.bf1 = (int)g.blk_f.size();
        // cells, ordered along a Morton curve, a Hilbert curve (the curve of the
        // paper's reorder, Sec. 2.2) through the enclosing 2^b cube, or x-fastest
        const int nc3 = nc * nc * nc;
        int bits = 1;
        while ((1 << bits) < nc)
            ++bits;
        std::vector<std::pair<uint32_t, int>> order(nc3);
        for (int lin = 0; lin < nc3; ++lin) {
            const int cx = lin % nc, cy = (lin / nc) % nc, cz = lin / (nc * nc);
            uint32_t code = (uint32_t)lin;
            if (p->reorder == 1)
                code = spread3(cx) | (spread3(cy) << 1) | (spread3(cz) << 2);
            else if (p->reorder == 2)
                code = hilbert3(cx, cy, cz, bits);
            order[lin] = {code, lin};
        }
        std::sort(order.begin(), order.end());
        g.crank.resize(cell0 + nc3);
        g.cxyz.resize(cell0 + nc3);
        for (int rank = 0; rank < nc3; ++rank) {
            const int lin = order[rank].second;
            g.crank[cell0 + lin] = cell0 + rank;
            g.cxyz[cell0 + rank] = make_int4(lin % nc, (lin / nc) % nc, lin / (nc * nc), r);
        }
        cell0 += nc3;
        g.n += nrep[r];
    }
    g.ncell = cell0;
    g.nblk_i = (int)g.blk_i.size();
    g.nblk_f = (int)g.blk_f.size();
    std::vector<double> bx(box, box + R);
    std::vector<int64_t> nr(nrep, nrep + R);
    g.K = p->neigh_capacity > 0 ? (p->neigh_capacity + 7) / 8 * 8 : auto_capacity(p, g, bx, nr);
    g.Kmax = p->neigh_capacity_max > 0 ? (p->neigh_capacity_max + 7) / 8 * 8 : 2 * g.K;
    if (g.Kmax < g.K) {
        msg = "neigh_capacity_max must be 0 or at least neigh_capacity";
        return MD_E_INVAL;
    }
    if ((double)g.n * (double)g.Kmax > 4.0e12) { msg = "neighbour-list cap too large"; return MD_E_INVAL; }
    g.check = p->check_interval > 0 ? p->check_interval : (g.n >= kCheckLargeN ? 1 : kCheck);
    return MD_OK;
}

Layout make_layout(const md_params *p, const Geometry &g)
{
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + std::max<size_t>(bytes, 1)); return r; };
    const size_t n = (size_t)g.n;
    const size_t pb = prec_pos_bytes(p->precision);
    const bool mixed = p->precision == MD_PREC_MIXED;
    const int cap = p->obs_capacity > 0 ? p->obs_capacity : 4096;
    L.off_ctl = take(sizeof(mdk::Ctl));
    L.off_rep = take(sizeof(mdk::Rep) * g.R);
    L.off_blk_i = take(sizeof(int4) * g.nblk_i);
    L.off_blk_f = take(sizeof(int4) * g.nblk_f);
    L.off_blk_s = take(sizeof(int4) * 2 * (size_t)g.nblk_f);   // < nblk_f + resident blocks rows
    L.off_crank = take(sizeof(int) * g.ncell);
    L.off_cxyz = take(sizeof(int4) * g.ncell);
    L.off_pa = take(pb * n);
    L.off_pb = take(mixed ? 16 * n : 0);
    L.off_va = take(pb * n);
    L.off_vb = take(mixed ? 16 * n : 0);
    L.off_pa2 = take(pb * n);
    L.off_pb2 = take(mixed ? 16 * n : 0);
    L.off_qa = take(mixed ? 16 * n : 0);
    L.off_qb = take(mixed ? 16 * n : 0);
    L.off_va2 = take(pb * n);
    L.off_vb2 = take(mixed ? 16 * n : 0);
    L.off_force = take(pb * n);
    L.off_rref = take(16 * n);
    L.off_image = take(16 * n);
    L.off_image2 = take(16 * n);
    L.off_key = take(4 * n);
    L.off_tmpidx = take(4 * n);
    L.off_skey = take(4 * n);
    L.off_ccount = take(4 * (size_t)g.ncell);
    L.off_ccursor = take(4 * (size_t)g.ncell);
    L.off_cstart = take(4 * ((size_t)g.ncell + 1));
    L.off_nbr = take(4 * n * (size_t)g.Kmax);       // room for the cap: K grows in place
    L.off_nnbr = take(4 * n);
    L.off_part_f = take(8 * 12 * (size_t)g.nblk_f);
    L.off_part_i = take(8 * 4 * (size_t)g.nblk_i);
    L.off_part_e = take(8 * 2 * (size_t)(kForceBlock / 32) * (size_t)g.nblk_f);   // per warp, 2 parities
    L.off_ring = take(sizeof(mdk::Obs) * (size_t)cap * g.R);
    L.off_epot = take(sizeof(double) * (size_t)cap * g.R);
    L.off_epot_step = take(sizeof(long long) * (size_t)cap);
    L.off_totals = take(sizeof(mdk::Obs) * g.R);
    L.off_scale = take(8 * (size_t)g.R);
    L.off_st_pos = take(24 * n);
    L.off_st_vel = take(24 * n);
    L.off_st_img = take(12 * n);
    L.off_st_code = take(4 * n);
    L.off_st_f = take(24 * n);
    L.off_st_e = take(8 * n);
    L.total = o;
    return L;
}

const KernelSet &kernel_set(int prec)
{
    if (prec == MD_PREC_FP64)
        return mdk::kernels_fp64();
    if (prec == MD_PREC_FP32)
        return mdk::kernels_fp32();
    return mdk::kernels_mixed();
}

int force_index(int tpp)
{
    int k = 0;
    while ((1 << k) < tpp)
        ++k;
    return k;
}

}  // namespace

struct md_handle {
    md_params p;
    Geometry g;
    Layout lay;
    cudaStream_t s = nullptr;
    char *ws = nullptr;
    KArgs a;
    const KernelSet *ks = nullptr;
    int cap = 4096;
    // pinned host staging
    char *pin = nullptr;
    size_t pin_bytes = 0;
    cudaEvent_t ev_stage = nullptr;
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    // timing of the force kernel (use_graph = 0)
    cudaEvent_t ev_f0 = nullptr, ev_f1 = nullptr, ev_i1 = nullptr;
    double step_ms = 0.0, rebuild_ms = 0.0;
    int64_t step_launches = 0, rebuild_checks = 0;
    int64_t obs_read = 0;
    int64_t epot_read = -1;          // newest step returned by md_epot_series
    int64_t n_species[2] = {0, 0};   // particles per species over all replicas
    std::string err;
};

namespace {

int fail(md_handle *h, int code, const std::string &m)
{
    if (h)
        h->err = m;
    return code;
}

int cuda_fail(md_handle *h, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, MD_E_CUDA, m);
}

#define CK(h, expr)                                   \
    do {                                              \
        cudaError_t e_ = (expr);                      \
        if (e_ != cudaSuccess)                        \
            return cuda_fail((h), e_, #expr);         \
    } while (0)

// The step kernel in use: lanes per particle, smoothing, and the block form.
const void *step_kernel(const md_handle *h)
{
    const int sm = h->p.smooth_h > 0.0, li = force_index(h->g.tpp);
    return h->g.sweep ? h->ks->step_sweep[sm][li] : h->ks->step[sm][li];
}

int launch(md_handle *h, const void *f, int grid, int block, const KArgs &a)
{
    if (grid <= 0)
        return MD_OK;
    void *pp[1] = {(void *)&a};
    CK(h, cudaLaunchKernel(f, dim3((unsigned)grid), dim3((unsigned)block), pp, 0, h->s));
    return MD_OK;
}

int grid_n(int64_t n, int per) { return (int)((n + per - 1) / per); }

// The rebuild chain: kernel, grid, block.
struct ChainStep { const void *f; int grid, block; };

// The neighbour build's kernel and launch shape: one warp per cell, kNbCells
// cells per block, unless the cells are too few to fill the GPU that way
// (fewer than one per resident warp slot), then one 8-warp block per cell.
ChainStep nbuild_step(const md_handle *h)
{
    if (h->g.nb_block)
        return {h->ks->nbuild_blk, h->g.ncell, kNbBlockB};
    return {h->ks->nbuild, (h->g.ncell + kNbCells - 1) / kNbCells, kNbBlock};
}

int rebuild_chain(const md_handle *h, ChainStep *seq)
{
    const KernelSet &k = *h->ks;
    const int nb = grid_n(h->g.n, kIntBlock);
    seq[0] = {k.bin, h->g.nblk_i, kIntBlock};
    seq[1] = {k.scan, 1, kScanBlock};
    seq[2] = {k.scatter, nb, kIntBlock};
    seq[3] = {k.permute, nb, kIntBlock};
    seq[4] = nbuild_step(h);                             // its last block makes
    return 5;                                            // the permuted buffers current or asks
}                                                        // for a redo with a larger K

// The redo of the build after its capacity grew: one block per cell as well.
KArgs retry_args(const md_handle *h)
{
    KArgs a = h->a;
    a.nb_retry = 1;
    return a;
}

// Stream launches of the chain; the redo is launched every time and returns at
// once unless the first build asked for it.
int launch_rebuild(md_handle *h)
{
    ChainStep seq[8];
    const int ns = rebuild_chain(h, seq);
    for (int s = 0; s < ns; ++s) {
        int rc = launch(h, seq[s].f, seq[s].grid, seq[s].block, h->a);
        if (rc)
            return rc;
    }
    const ChainStep nb = nbuild_step(h);
    return launch(h, nb.f, nb.grid, nb.block, retry_args(h));
}

// Arguments of the step kernel at position `slot` of the unrolled loop.
KArgs step_args(const md_handle *h, int slot)
{
    KArgs a = h->a;
    a.imode = mdk::IM_LOOP;
    const int ci = h->g.check;
    const bool check = (slot % ci) == ci - 1;
    a.lookahead = check ? ci - 1 : 0;
    a.set_rebuild = check ? 1 : 0;
    a.set_loop = slot == kUnroll - 1 ? 1 : 0;
    return a;
}

KArgs first_args(const md_handle *h)
{
    KArgs a = h->a;
    a.imode = mdk::IM_FIRST;
    a.lookahead = h->g.check - 1;
    a.set_rebuild = 1;
    return a;
}

// Energies of a step still awaiting their sum go into the per-step series
// first: the force kernel reuses the partials' storage.
int flush_epot(md_handle *h) { return launch(h, h->ks->epot_flush, 1, kForceBlock, h->a); }

int launch_force(md_handle *h, int fsample)
{
    KArgs a = h->a;
    a.fsample = fsample;
    int rc = flush_epot(h);
    if (rc)
        return rc;
    return launch(h, h->ks->force[h->p.smooth_h > 0.0][force_index(h->g.tpp)], h->g.nblk_f, kForceBlock, a);
}

int launch_integrate(md_handle *h, int mode)
{
    KArgs a = h->a;
    a.imode = mode;
    a.use_cond = 0;
    return launch(h, h->ks->integrate, h->g.nblk_i, kIntBlock, a);
}

// ---- graph construction ----
int add_kernel(md_handle *h, cudaGraph_t g, cudaGraphNode_t *node, const cudaGraphNode_t *deps, size_t ndeps,
               const void *f, int grid, int block, const KArgs &a)
{
    alignas(cudaGraphNodeParams) unsigned char np_buf[sizeof(cudaGraphNodeParams)] = {};
    cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(np_buf);
    np.type = cudaGraphNodeTypeKernel;
    np.kernel.func = (void *)f;
    np.kernel.gridDim = dim3((unsigned)grid);
    np.kernel.blockDim = dim3((unsigned)block);
    np.kernel.sharedMemBytes = 0;
    void *pp[1] = {(void *)&a};
    np.kernel.kernelParams = pp;
    CK(h, cudaGraphAddNode(node, g, deps, nullptr, ndeps, &np));
    return MD_OK;
}

int add_conditional(md_handle *h, cudaGraph_t g, cudaGraphNode_t *node, cudaGraphNode_t dep,
                    cudaGraphConditionalHandle c, cudaGraphConditionalNodeType type, cudaGraph_t *body);

// The rebuild chain as graph nodes, closed by a conditional redo of the build
// that runs only when the build grew the list capacity.
int add_rebuild_chain(md_handle *h, cudaGraph_t g)
{
    ChainStep seq[8];
    const int ns = rebuild_chain(h, seq);
    cudaGraphConditionalHandle c_regrow;
    CK(h, cudaGraphConditionalHandleCreate(&c_regrow, g, 0, 0));
    cudaGraphNode_t prev = nullptr;
    for (int s = 0; s < ns; ++s) {
        cudaGraphNode_t node;
        KArgs a = h->a;
        if (s == ns - 1) {                              // the build
            a.use_cond = 1;
            a.set_regrow = 1;
            a.h_regrow = c_regrow;
        }
        int rc = add_kernel(h, g, &node, prev ? &prev : nullptr, prev ? 1 : 0, seq[s].f, seq[s].grid,
                            seq[s].block, a);
        if (rc)
            return rc;
        prev = node;
    }
    cudaGraphNode_t n_if;
    cudaGraph_t body;
    int rc = add_conditional(h, g, &n_if, prev, c_regrow, cudaGraphCondTypeIf, &body);
    if (rc)
        return rc;
    cudaGraphNode_t n_retry;
    const ChainStep nb = nbuild_step(h);
    return add_kernel(h, body, &n_retry, nullptr, 0, nb.f, nb.grid, nb.block, retry_args(h));
}

int add_conditional(md_handle *h, cudaGraph_t g, cudaGraphNode_t *node, cudaGraphNode_t dep,
                    cudaGraphConditionalHandle c, cudaGraphConditionalNodeType type, cudaGraph_t *body)
{
    alignas(cudaGraphNodeParams) unsigned char np_buf[sizeof(cudaGraphNodeParams)] = {};
    cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(np_buf);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = c;
    np.conditional.type = type;
    np.conditional.size = 1;
    CK(h, cudaGraphAddNode(node, g, &dep, nullptr, 1, &np));
    *body = np.conditional.phGraph_out[0];
    return MD_OK;
}

int build_graph(md_handle *h)
{
    int rc;
    cudaGraph_t g;
    CK(h, cudaGraphCreate(&g, 0));
    h->graph = g;
    cudaGraphConditionalHandle c_loop, c_reb0;
    CK(h, cudaGraphConditionalHandleCreate(&c_loop, g, 1, cudaGraphCondAssignDefault));
    CK(h, cudaGraphConditionalHandleCreate(&c_reb0, g, 0, 0));

    KArgs first = first_args(h);
    first.use_cond = 1;
    first.h_rebuild = c_reb0;
    first.h_loop = c_loop;
    cudaGraphNode_t n_first, n_if0, n_while;
    if ((rc = add_kernel(h, g, &n_first, nullptr, 0, h->ks->integrate, h->g.nblk_i, kIntBlock, first)))
        return rc;
    cudaGraph_t body0;
    if ((rc = add_conditional(h, g, &n_if0, n_first, c_reb0, cudaGraphCondTypeIf, &body0)))
        return rc;
    if ((rc = add_rebuild_chain(h, body0)))
        return rc;
    cudaGraph_t wbody;
    if ((rc = add_conditional(h, g, &n_while, n_if0, c_loop, cudaGraphCondTypeWhile, &wbody)))
        return rc;
    // loop body: kUnroll step kernels, a conditional rebuild after every g.check
    const void *stepk = step_kernel(h);
    cudaGraphNode_t prev = nullptr;
    for (int slot = 0; slot < kUnroll; ++slot) {
        KArgs sa = step_args(h, slot);
        sa.use_cond = 1;
        sa.h_loop = c_loop;
        cudaGraphConditionalHandle c_reb = 0;
        if (sa.set_rebuild) {
            CK(h, cudaGraphConditionalHandleCreate(&c_reb, wbody, 0, 0));
            sa.h_rebuild = c_reb;
        }
        cudaGraphNode_t n_s;
        if ((rc = add_kernel(h, wbody, &n_s, prev ? &prev : nullptr, prev ? 1 : 0, stepk, h->g.nblk_s,
                             kForceBlock, sa)))
            return rc;
        prev = n_s;
        if (sa.set_rebuild) {
            cudaGraphNode_t n_if;
            cudaGraph_t body;
            if ((rc = add_conditional(h, wbody, &n_if, n_s, c_reb, cudaGraphCondTypeIf, &body)))
                return rc;
            if ((rc = add_rebuild_chain(h, body)))
                return rc;
            prev = n_if;
        }
    }
    CK(h, cudaGraphInstantiate(&h->gexec, g, 0));
    return MD_OK;
}

int stage_wait(md_handle *h)
{
    CK(h, cudaEventSynchronize(h->ev_stage));
    return MD_OK;
}

int ensure_pinned(md_handle *h, size_t bytes)
{
    if (bytes <= h->pin_bytes)
        return MD_OK;
    int rc = stage_wait(h);
    if (rc)
        return rc;
    CK(h, cudaStreamSynchronize(h->s));
    if (h->pin)
        cudaFreeHost(h->pin);
    h->pin = nullptr;
    h->pin_bytes = 0;
    CK(h, cudaMallocHost((void **)&h->pin, bytes));
    h->pin_bytes = bytes;
    return MD_OK;
}

int read_ctl(md_handle *h, mdk::Ctl *out)
{
    int rc = ensure_pinned(h, sizeof(mdk::Ctl));
    if (rc)
        return rc;
    if ((rc = stage_wait(h)))
        return rc;
    CK(h, cudaMemcpyAsync(h->pin, h->a.ctl, sizeof(mdk::Ctl), cudaMemcpyDeviceToHost, h->s));
    CK(h, cudaStreamSynchronize(h->s));
    memcpy(out, h->pin, sizeof(mdk::Ctl));
    return MD_OK;
}

// Stream-launch mode: launch the rebuild chain if the device flag asks for it
// (waits for the stream); adds its CUDA-event time to *ms when given.
int rebuild_if_flagged(md_handle *h, float *ms)
{
    mdk::Ctl c;
    int rc = read_ctl(h, &c);
    if (rc)
        return rc;
    if (!c.rebuild || c.status)
        return MD_OK;
    CK(h, cudaEventRecord(h->ev_f1, h->s));
    if ((rc = launch_rebuild(h)))
        return rc;
    CK(h, cudaEventRecord(h->ev_i1, h->s));
    CK(h, cudaEventSynchronize(h->ev_i1));
    if (ms)
        CK(h, cudaEventElapsedTime(ms, h->ev_f1, h->ev_i1));
    h->rebuild_checks += 1;
    return MD_OK;
}

int status_code(unsigned st)
{
    if (st & mdk::ST_NONFINITE) return MD_E_NONFINITE;
    if (st & mdk::ST_UNSTABLE) return MD_E_UNSTABLE;
    if (st & mdk::ST_OVERFLOW) return MD_E_CAPACITY;
    if (st & mdk::ST_TIMEOUT) return MD_E_TIMEOUT;
    if (st & mdk::ST_BOUNDS) return MD_E_BOUNDS;
    return MD_OK;
}

const char *status_message(int code)
{
    switch (code) {
    case MD_E_NONFINITE: return "a position became non-finite; the step loop stopped";
    case MD_E_UNSTABLE: return "a particle moved more than a quarter box in one step; the step loop stopped";
    case MD_E_CAPACITY: return "a neighbour list exceeded neigh_capacity_max; the step loop stopped";
    case MD_E_BOUNDS: return "an index left its array (bounds-checked build); the access was redirected";
    case MD_E_TIMEOUT: return "the device step loop exceeded its iteration bound";
    default: return "";
    }
}

// Synchronise, report (once) and clear a device status.
int check_device(md_handle *h)
{
    mdk::Ctl c;
    int rc = read_ctl(h, &c);
    if (rc)
        return rc;
    const int code = status_code(c.status);
    if (code != MD_OK) {
        KArgs a = h->a;
        if ((rc = launch(h, h->ks->reset, 1, 1, a)))
            return rc;
        CK(h, cudaStreamSynchronize(h->s));
        return fail(h, code, status_message(code));
    }
    return MD_OK;
}

// Copy the caller's state into pinned staging, upload it, load it into the
// working layout, rebuild, evaluate forces.
int upload_state(md_handle *h, const int32_t *species, const double *pos, const double *vel,
                 const int32_t *image)
{
    const size_t n = (size_t)h->g.n;
    const size_t bytes = 24 * n + 24 * n + 12 * n + 4 * n;
    int rc = ensure_pinned(h, bytes);
    if (rc)
        return rc;
    if ((rc = stage_wait(h)))
        return rc;
    char *q = h->pin;
    memcpy(q, pos, 24 * n);
    if (vel)
        memcpy(q + 24 * n, vel, 24 * n);
    else
        memset(q + 24 * n, 0, 24 * n);
    if (image)
        memcpy(q + 48 * n, image, 12 * n);
    else
        memset(q + 48 * n, 0, 12 * n);
    memcpy(q + 60 * n, species, 4 * n);
    CK(h, cudaMemcpyAsync(h->a.st_pos, q, 24 * n, cudaMemcpyHostToDevice, h->s));
    CK(h, cudaMemcpyAsync(h->a.st_vel, q + 24 * n, 24 * n, cudaMemcpyHostToDevice, h->s));
    CK(h, cudaMemcpyAsync(h->a.st_img, q + 48 * n, 12 * n, cudaMemcpyHostToDevice, h->s));
    CK(h, cudaMemcpyAsync(h->a.st_code, q + 60 * n, 4 * n, cudaMemcpyHostToDevice, h->s));
    CK(h, cudaEventRecord(h->ev_stage, h->s));
    if ((rc = launch(h, h->ks->load, h->g.nblk_i, kIntBlock, h->a)))
        return rc;
    if ((rc = launch_rebuild(h)))
        return rc;
    return launch_force(h, 1);
}

}  // namespace

extern "C" {

int md_params_default(md_params *p)
{
    if (!p)
        return MD_E_INVAL;
    memset(p, 0, sizeof *p);
    p->n_species = 1;
    p->shift = 1;
    for (int a = 0; a < 2; ++a) {
        for (int b = 0; b < 2; ++b) {
            p->eps[a][b] = 1.0;
            p->sigma[a][b] = 1.0;
            p->rcut[a][b] = 2.5;
        }
        p->mass[a] = 1.0;
    }
    p->dt = 0.005;
    p->skin = 0.3;
    p->precision = MD_PREC_MIXED;
    p->sample_interval = 100;
    p->use_graph = 1;
    p->reorder = 1;
    return MD_OK;
}

int md_cell_order(const md_params *p, int32_t n_replicas, const int64_t *n_per_replica, const double *box,
                  int32_t *rank, int32_t *cells_per_edge)
{
    Geometry g;
    std::string msg;
    int rc = make_geometry(p, n_replicas, n_per_replica, box, g, msg);
    if (rc)
        return rc;
    const int nc = g.rep[0].nc;
    if (cells_per_edge)
        *cells_per_edge = nc;
    if (rank)
        for (int lin = 0; lin < nc * nc * nc; ++lin)
            rank[lin] = g.crank[lin];
    return MD_OK;
}

int md_workspace_size(const md_params *p, int32_t n_replicas, const int64_t *n_per_replica,
                      const double *box, size_t *bytes)
{
    if (!bytes)
        return MD_E_INVAL;
    Geometry g;
    std::string msg;
    int rc = make_geometry(p, n_replicas, n_per_replica, box, g, msg);
    if (rc)
        return rc;
    *bytes = make_layout(p, g).total;
    return MD_OK;
}

static int create_impl(md_handle *h, const md_params *p, const int32_t *species, const double *pos,
                       const double *vel, const int32_t *image, void *workspace, size_t workspace_bytes,
                       void *cuda_stream)
{
    int rc;
    h->p = *p;
    h->lay = make_layout(p, h->g);
    if (!species || !pos || !workspace || ((uintptr_t)workspace % kAlign) != 0)
        return fail(h, MD_E_INVAL, "null array or workspace not 256-byte aligned");
    if (workspace_bytes < h->lay.total)
        return fail(h, MD_E_NOMEM, "workspace smaller than md_workspace_size()");
    for (int64_t i = 0; i < h->g.n; ++i)
        if (species[i] < 0 || species[i] >= p->n_species)
            return fail(h, MD_E_INVAL, "species out of range");
    for (int64_t i = 0; i < h->g.n; ++i)
        h->n_species[species[i]] += 1;
    for (auto &q : h->g.rep) {
        double m = 0.0;
        for (int i = q.start; i < q.start + q.n; ++i)
            m += p->mass[species[i]];
        q.mtot = m;
    }
    h->s = (cudaStream_t)cuda_stream;
    h->ws = (char *)workspace;
    h->ks = &kernel_set(p->precision);
    h->cap = p->obs_capacity > 0 ? p->obs_capacity : 4096;
    const Geometry &g = h->g;
    const Layout &L = h->lay;
    KArgs &a = h->a;
    memset(&a, 0, sizeof a);
    char *w = h->ws;
    a.n = (int)g.n;
    a.nrep = g.R;
    a.ncell = g.ncell;
    a.Kstride = g.Kmax;
    a.tpp = g.tpp;
    a.si = p->sample_interval;
    a.obs_cap = h->cap;
    a.epot_cap = h->cap;
    a.nblk_i = g.nblk_i;
    a.nblk_f = g.nblk_f;
    a.pa = w + L.off_pa; a.pb = w + L.off_pb; a.va = w + L.off_va; a.vb = w + L.off_vb;
    a.pa2 = w + L.off_pa2; a.pb2 = w + L.off_pb2; a.va2 = w + L.off_va2; a.vb2 = w + L.off_vb2;
    a.qa = (int4 *)(w + L.off_qa); a.qb = (int4 *)(w + L.off_qb);
    a.force = w + L.off_force;
    a.rref = (float4 *)(w + L.off_rref);
    a.image = (int4 *)(w + L.off_image);
    a.image2 = (int4 *)(w + L.off_image2);
    a.key = (int *)(w + L.off_key);
    a.tmpidx = (int *)(w + L.off_tmpidx);
    a.skey = (int *)(w + L.off_skey);
    a.ccount = (int *)(w + L.off_ccount);
    a.ccursor = (int *)(w + L.off_ccursor);
    a.cstart = (int *)(w + L.off_cstart);
    a.crank = (const int *)(w + L.off_crank);
    a.cxyz = (const int4 *)(w + L.off_cxyz);
    a.nbr = (int *)(w + L.off_nbr);
    a.nnbr = (int *)(w + L.off_nnbr);
    a.blk_i = (const int4 *)(w + L.off_blk_i);
    a.blk_f = (const int4 *)(w + L.off_blk_f);
    a.blk_s = (const int4 *)(w + L.off_blk_s);
    a.cpb = g.cpb;
    a.part_f = (double *)(w + L.off_part_f);
    a.part_i = (double *)(w + L.off_part_i);
    a.part_e = w + L.off_part_e;
    a.ring = (mdk::Obs *)(w + L.off_ring);
    a.epot = (double *)(w + L.off_epot);
    a.epot_step = (long long *)(w + L.off_epot_step);
    a.totals = (mdk::Obs *)(w + L.off_totals);
    a.ctl = (mdk::Ctl *)(w + L.off_ctl);
    a.rep = (const mdk::Rep *)(w + L.off_rep);
    a.st_pos = (double *)(w + L.off_st_pos);
    a.st_vel = (double *)(w + L.off_st_vel);
    a.st_img = (int *)(w + L.off_st_img);
    a.st_code = (int *)(w + L.off_st_code);
    a.st_f = (double *)(w + L.off_st_f);
    a.st_e = (double *)(w + L.off_st_e);
    a.scale = (double *)(w + L.off_scale);
    // pair table (Sec. 3 potential, Sec. 5 parameters)
    for (int x = 0; x < 2; ++x)
        for (int y = 0; y < 2; ++y) {
            const int k = x * 2 + y;
            const int xs = std::min(x, p->n_species - 1), ys = std::min(y, p->n_species - 1);
            const double eps = p->eps[xs][ys], sig = p->sigma[xs][ys], rc = p->rcut[xs][ys];
            const double sr6 = std::pow(sig / rc, 6.0);
            const double shift = p->shift ? 4.0 * eps * (sr6 * sr6 - sr6) : 0.0;
            const double rl = rc + p->skin + (double)mdk::kListMargin;
            a.tab.rc2d[k] = rc * rc;
            a.tab.rl2d[k] = rl * rl;
            a.tab.sig2d[k] = sig * sig;
            a.tab.eps4d[k] = 4.0 * eps;
            a.tab.eps48d[k] = 48.0 * eps;
            a.tab.shiftd[k] = shift;
            a.tab.rc2[k] = (float)(rc * rc);
            a.tab.rl2[k] = (float)(rl * rl);
            a.tab.sig2[k] = (float)(sig * sig);
            a.tab.eps4[k] = (float)(4.0 * eps);
            a.tab.eps48[k] = (float)(48.0 * eps);
            a.tab.shift[k] = (float)shift;
            // smoothing of Sec. 4: x = (r - r_c) / (h sigma_ab)
            const double ihs = p->smooth_h > 0.0 ? 1.0 / (p->smooth_h * sig) : 0.0;
            a.tab.rcd[k] = rc;
            a.tab.ihsd[k] = ihs;
            a.tab.rc[k] = (float)rc;
            a.tab.ihs[k] = (float)ihs;
            a.tab.vcd[k] = eps != 0.0 ? shift / (4.0 * eps) : 0.0;
            a.tab.vc[k] = (float)a.tab.vcd[k];
        }
    for (int s = 0; s < 2; ++s) {
        const int ss = std::min(s, p->n_species - 1);
        const double m = p->mass[ss];
        const double hk = 0.5 * p->dt / m;
        a.mass[s] = m;
        a.hdtm[s] = hk;
        a.hdtm_hi[s] = (float)hk;
        a.hdtm_lo[s] = (float)(hk - (double)(float)hk);
    }
    a.dt = p->dt;
    a.dt_hi = (float)p->dt;
    a.dt_lo = (float)(p->dt - (double)(float)p->dt);
    const double thr = std::max(0.5 * p->skin - (double)mdk::kDispMargin, 0.0);
    a.disp_thr2 = (float)(thr * thr);
    a.disp_thr = (float)thr;
    for (int s = 0; s < 2; ++s)
        a.inv_mass[s] = (float)(1.0 / a.mass[s]);
    if (a.hdtm_hi[0] == 0.0f)
        return fail(h, MD_E_INVAL, "dt / (2 m) underflows single precision");

    int dev = 0, nsm = 0, per_sm = 0, per_sm_sw = 0;
    CK(h, cudaGetDevice(&dev));
    CK(h, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    {
        // step kernel: the sweeping form when asked for, or (automatic) when one block per chunk
        // would need more blocks than the GPU holds at once
        const int sm = h->p.smooth_h > 0.0, li = force_index(g.tpp);
        const void *sweepk = li < 2 ? h->ks->step_sweep[sm][li] : nullptr;
        CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, h->ks->step[sm][li], kForceBlock, 0));
        if (sweepk)
            CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_sw, sweepk, kForceBlock, 0));
        h->g.sweep = sweepk && per_sm_sw > 0 &&
                     (p->step_form == 2 || (p->step_form == 0 && (int64_t)g.nblk_f > (int64_t)nsm * per_sm_sw));
    }
    // the build takes a warp per cell when there are at least kNbWarpCellsPerSm cells per SM
    // and a cell's particles fit one batch of lanes on average; a block per cell otherwise
    // (measured on GB300: LJ at 729 cells or fewer and dense cells of ~40 are faster with a
    // block per cell, LJ from 1331 cells and KA N=65,536 with a warp per cell)
    h->g.nb_block = p->build_form == 2 ||
                    (p->build_form == 0 && ((int64_t)g.ncell < (int64_t)kNbWarpCellsPerSm * nsm ||
                                            (double)g.n > 32.0 * (double)g.ncell));
    // pinned staging, events
    CK(h, cudaEventCreateWithFlags(&h->ev_stage, cudaEventDisableTiming));
    CK(h, cudaEventCreate(&h->ev_f0));
    CK(h, cudaEventCreate(&h->ev_f1));
    CK(h, cudaEventCreate(&h->ev_i1));
    CK(h, cudaEventRecord(h->ev_stage, h->s));
    size_t tbytes = sizeof(mdk::Rep) * g.R + sizeof(int4) * (g.nblk_i + 3 * (size_t)g.nblk_f) +
                    sizeof(int) * g.ncell + sizeof(int4) * g.ncell;
    size_t sbytes = 64 * (size_t)g.n;
    if ((rc = ensure_pinned(h, std::max(tbytes, sbytes) + 4096)))
        return rc;
    // tables
    {
        char *q = h->pin;
        auto put = [&](size_t off, const void *src, size_t bytes) -> int {
            memcpy(q, src, bytes);
            cudaError_t e = cudaMemcpyAsync(w + off, q, bytes, cudaMemcpyHostToDevice, h->s);
            q += align_up(bytes);
            return e == cudaSuccess ? MD_OK : cuda_fail(h, e, "table upload");
        };
        const std::vector<int4> bf = mdt::sm_block_order(g.blk_f, nsm, nsm * per_sm);
        const std::vector<int4> bs =
            mdt::step_table(bf, g.blk_f, h->g.sweep, nsm, per_sm_sw, h->g.nblk_s, h->g.cpb);
        h->a.cpb = h->g.cpb;
        if ((rc = put(L.off_rep, g.rep.data(), sizeof(mdk::Rep) * g.R)) ||
            (rc = put(L.off_blk_i, g.blk_i.data(), sizeof(int4) * g.nblk_i)) ||
            (rc = put(L.off_blk_f, bf.data(), sizeof(int4) * g.nblk_f)) ||
            (rc = put(L.off_blk_s, bs.data(), sizeof(int4) * bs.size())) ||
            (rc = put(L.off_crank, g.crank.data(), sizeof(int) * g.ncell)) ||
            (rc = put(L.off_cxyz, g.cxyz.data(), sizeof(int4) * g.ncell)))
            return rc;
        mdk::Ctl c0;
        memset(&c0, 0, sizeof c0);
        c0.K = g.K;
        c0.Kmax = g.Kmax;
        c0.epot_pending = -1;
        if ((rc = put(L.off_ctl, &c0, sizeof c0)))
            return rc;
        cudaError_t e = cudaMemsetAsync(a.ccount, 0, 4 * (size_t)g.ncell, h->s);
        if (e == cudaSuccess)   // every slot of the per-step series empty (step -1)
            e = cudaMemsetAsync(a.epot_step, 0xff, sizeof(long long) * (size_t)h->cap, h->s);
        if (e == cudaSuccess)
            e = cudaEventRecord(h->ev_stage, h->s);
        if (e != cudaSuccess)
            return cuda_fail(h, e, "initialisation");
    }
    if ((rc = upload_state(h, species, pos, vel, image)) || (rc = launch_integrate(h, mdk::IM_SAMPLE)))
        return rc;
    return check_device(h);
}

int md_create(md_handle **out, const md_params *p, int32_t n_replicas, const int64_t *n_per_replica,
              const double *box, const int32_t *species, const double *pos, const double *vel,
              const int32_t *image, void *workspace, size_t workspace_bytes, void *cuda_stream)
{
    ApiRange range_("md_create");
    if (!out)
        return MD_E_INVAL;
    *out = nullptr;
    md_handle *h = new (std::nothrow) md_handle();
    if (!h)
        return MD_E_NOMEM;
    std::string msg;
    int rc = make_geometry(p, n_replicas, n_per_replica, box, h->g, msg);
    if (rc == MD_OK)
        rc = create_impl(h, p, species, pos, vel, image, workspace, workspace_bytes, cuda_stream);
    if (rc != MD_OK) {
        md_destroy(h);
        return rc;
    }
    *out = h;
    return MD_OK;
}

int md_step(md_handle *h, int64_t nsteps)
{
    ApiRange range_("md_step");
    if (!h)
        return MD_E_INVAL;
    if (nsteps < 1)
        return fail(h, MD_E_INVAL, "nsteps must be >= 1");
    int rc;
    KArgs a = h->a;
    a.nsteps = nsteps;
    a.budget = h->p.step_budget;
    if ((rc = launch(h, h->ks->set_steps, 1, 1, a)))
        return rc;
    if (h->p.use_graph) {
        if (!h->gexec && (rc = build_graph(h)))
            return rc;
        CK(h, cudaGraphLaunch(h->gexec, h->s));
        return MD_OK;
    }
    // The graph's kernel sequence, launched from the host with per-kernel
    // timing.  At each check point the host reads the device's rebuild flag
    // and launches the rebuild chain only when the graph's IF node would run
    // it, so exactly the same kernels execute (results are bitwise equal).
    if ((rc = launch(h, h->ks->integrate, h->g.nblk_i, kIntBlock, first_args(h))) ||
        (rc = rebuild_if_flagged(h, nullptr)))
        return rc;
    const void *stepk = step_kernel(h);
    const int64_t iters = (nsteps + kUnroll - 1) / kUnroll;
    for (int64_t it = 0; it < iters; ++it) {
        for (int slot = 0; slot < kUnroll; ++slot) {
            const KArgs sa = step_args(h, slot);
            CK(h, cudaEventRecord(h->ev_f0, h->s));
            if ((rc = launch(h, stepk, h->g.nblk_s, kForceBlock, sa)))
                return rc;
            CK(h, cudaEventRecord(h->ev_f1, h->s));
            CK(h, cudaEventSynchronize(h->ev_f1));
            float ms = 0.f;
            CK(h, cudaEventElapsedTime(&ms, h->ev_f0, h->ev_f1));
            if (it * kUnroll + slot < nsteps) {
                h->step_ms += ms;
                h->step_launches += 1;
            }
            if (sa.set_rebuild) {
                float mr = 0.f;
                if ((rc = rebuild_if_flagged(h, &mr)))
                    return rc;
                h->rebuild_ms += mr;
            }
        }
    }
    return MD_OK;
}

int md_rescale_velocities(md_handle *h, const double *T_target)
{
    ApiRange range_("md_rescale_velocities");
    if (!h || !T_target)
        return MD_E_INVAL;
    int rc;
    for (int r = 0; r < h->g.R; ++r)
        if (!(T_target[r] >= 0.0))
            return fail(h, MD_E_INVAL, "target temperatures must be >= 0");
    if ((rc = stage_wait(h)))
        return rc;
    memcpy(h->pin, T_target, 8 * (size_t)h->g.R);
    CK(h, cudaMemcpyAsync(h->a.scale, h->pin, 8 * (size_t)h->g.R, cudaMemcpyHostToDevice, h->s));
    CK(h, cudaEventRecord(h->ev_stage, h->s));
    if ((rc = launch_integrate(h, mdk::IM_KE)))
        return rc;
    return launch(h, h->ks->scale, h->g.nblk_i, kIntBlock, h->a);
}

// Andersen heat bath (Sec. 2.3): one collision of every particle.
int md_andersen(md_handle *h, const double *T_target, uint64_t seed, int64_t event)
{
    ApiRange range_("md_andersen");
    if (!h || !T_target)
        return MD_E_INVAL;
    if (event < 0)
        return fail(h, MD_E_INVAL, "event index must be >= 0");
    const unsigned long long n = (unsigned long long)h->g.n;
    if ((unsigned long long)event > (~0ull >> 1) / 4 / (n + 1))
        return fail(h, MD_E_INVAL, "event index too large");
    int rc;
    for (int r = 0; r < h->g.R; ++r)
        if (!(T_target[r] >= 0.0) || !std::isfinite(T_target[r]))
            return fail(h, MD_E_INVAL, "target temperatures must be finite and >= 0");
    if ((rc = stage_wait(h)))
        return rc;
    memcpy(h->pin, T_target, 8 * (size_t)h->g.R);
    CK(h, cudaMemcpyAsync(h->a.scale, h->pin, 8 * (size_t)h->g.R, cudaMemcpyHostToDevice, h->s));
    CK(h, cudaEventRecord(h->ev_stage, h->s));
    // rand48 (a = 0x5DEECE66D, c = 0xB, modulo 2^48), seeded as srand48; leapfrog over n threads
    const unsigned long long A = 0x5DEECE66DULL, Cc = 0xBULL, mask = 0xFFFFFFFFFFFFULL;
    unsigned long long AN = 1, CN = 0, Ab = A, Cb = Cc;
    for (unsigned long long p = n; p; p >>= 1) {
        if (p & 1ull) {
            AN = (Ab * AN) & mask;
            CN = (Ab * CN + Cb) & mask;
        }
        Cb = (Ab * Cb + Cb) & mask;
        Ab = (Ab * Ab) & mask;
    }
    mdk::KArgs a = h->a;
    a.r48_x0 = ((seed & 0xFFFFFFFFull) << 16) | 0x330Eull;
    a.r48_AN = AN;
    a.r48_CN = CN;
    a.r48_base = (long long)(4ull * (unsigned long long)event * n);
    if ((rc = launch(h, h->ks->andersen, h->g.nblk_i, kIntBlock, a)) ||
        (rc = launch_integrate(h, mdk::IM_TOTALS)))
        return rc;
    return launch(h, h->ks->andersen_fix, h->g.nblk_i, kIntBlock, h->a);
}

// ---------------------------------------------------------------------------
// Blocking scheme for time-correlation functions (Sec. 2.5).  Block n holds at
// most l samples spaced l^n samples apart; when it is full its first entry is
// correlated with the others and dropped.  Snapshots live in a pool of k l
// slots shared by the blocks (a sample that enters several blocks is stored
// once); the host keeps the bookkeeping, the device the data and the sums.
// ---------------------------------------------------------------------------
struct md_corr {
    md_handle *h = nullptr;
    int k = 0, l = 0, nq = 0, nblocks = 0;
    int64_t m = 0;                            // samples taken
    double *pool = nullptr;                   // [k l][n][3]
    int *species = nullptr;                   // [n]
    double *q = nullptr;                      // [nq][3]
    double *part = nullptr;                   // [nblocks][l-1][4]
    double *acc = nullptr;                    // [k][l-1][4]
    std::vector<std::vector<int>> blocks;     // slot ids, oldest first
    std::vector<int> refs;                    // blocks referring to each slot
    std::vector<int64_t> origins;             // [k][l-1]
};

namespace {

size_t corr_layout(int64_t n, int k, int l, int nq, size_t off[6])
{
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + std::max<size_t>(bytes, 1)); return r; };
    const size_t nb = (size_t)((n + mdk::kCorrBlock - 1) / mdk::kCorrBlock);
    off[0] = take(sizeof(double) * 3 * (size_t)n * (size_t)k * (size_t)l);
    off[1] = take(sizeof(int) * (size_t)n);
    off[2] = take(sizeof(double) * 3 * (size_t)nq);
    off[3] = take(sizeof(double) * 4 * nb * (size_t)(l - 1));
    off[4] = take(sizeof(double) * 4 * (size_t)k * (size_t)(l - 1));
    off[5] = o;
    return o;
}

int corr_check(const md_handle *h, int k, int l, int nq)
{
    if (!h || k < 1 || l < 2 || l - 1 > mdk::kCorrMaxJ || nq < 1 || nq > mdk::kCorrMaxQ)
        return MD_E_INVAL;
    double span = 1.0;                         // l^k must stay a valid sample index
    for (int n = 0; n < k; ++n)
        span *= l;
    return span < 9e15 ? MD_OK : MD_E_INVAL;
}

}  // namespace

int md_corr_workspace_size(const md_handle *h, int32_t k, int32_t l, int32_t n_q, size_t *bytes)
{
    if (!bytes || corr_check(h, k, l, n_q))
        return MD_E_INVAL;
    size_t off[6];
    *bytes = corr_layout(h->g.n, k, l, n_q, off);
    return MD_OK;
}

int md_corr_create(md_corr **out, md_handle *h, int32_t k, int32_t l, int32_t n_q, const double *q,
                   void *workspace, size_t workspace_bytes)
{
    ApiRange range_("md_corr_create");
    if (!out || !q || corr_check(h, k, l, n_q))
        return h ? fail(h, MD_E_INVAL, "md_corr_create: bad arguments (1 <= k, 2 <= l <= 32, "
                                       "1 <= n_q <= 64, non-null q)") : MD_E_INVAL;
    *out = nullptr;
    size_t off[6];
    const size_t need = corr_layout(h->g.n, k, l, n_q, off);
    if (!workspace || ((uintptr_t)workspace % kAlign) != 0)
        return fail(h, MD_E_INVAL, "md_corr_create: workspace missing or not 256-byte aligned");
    if (workspace_bytes < need)
        return fail(h, MD_E_NOMEM, "md_corr_create: workspace smaller than md_corr_workspace_size()");
    for (int t = 0; t < 3 * n_q; ++t)
        if (!std::isfinite(q[t]))
            return fail(h, MD_E_INVAL, "md_corr_create: non-finite wavevector");
    md_corr *c = new (std::nothrow) md_corr;
    if (!c)
        return fail(h, MD_E_NOMEM, "md_corr_create: host allocation failed");
    char *w = (char *)workspace;
    c->h = h;
    c->k = k;
    c->l = l;
    c->nq = n_q;
    c->nblocks = (int)((h->g.n + mdk::kCorrBlock - 1) / mdk::kCorrBlock);
    c->pool = (double *)(w + off[0]);
    c->species = (int *)(w + off[1]);
    c->q = (double *)(w + off[2]);
    c->part = (double *)(w + off[3]);
    c->acc = (double *)(w + off[4]);
    c->blocks.assign(k, std::vector<int>());
    c->refs.assign((size_t)k * l, 0);
    c->origins.assign((size_t)k * (l - 1), 0);
    int rc;
    if ((rc = stage_wait(h)) || (rc = ensure_pinned(h, sizeof(double) * 3 * n_q))) {
        delete c;
        return rc;
    }
    memcpy(h->pin, q, sizeof(double) * 3 * n_q);
    cudaError_t e = cudaMemcpyAsync(c->q, h->pin, sizeof(double) * 3 * n_q, cudaMemcpyHostToDevice, h->s);
    if (e == cudaSuccess)
        e = cudaEventRecord(h->ev_stage, h->s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->acc, 0, sizeof(double) * 4 * (size_t)k * (l - 1), h->s);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(h, e, "md_corr_create");
    }
    *out = c;
    return MD_OK;
}

int md_corr_sample(md_corr *c)
{
    ApiRange range_("md_corr_sample");
    if (!c)
        return MD_E_INVAL;
    md_handle *h = c->h;
    int slot = -1;
    for (size_t s = 0; s < c->refs.size(); ++s)
        if (c->refs[s] == 0) {
            slot = (int)s;
            break;
        }
    if (slot < 0)
        return fail(h, MD_E_INVAL, "md_corr_sample: no free snapshot slot");   // cannot happen: k l slots
    const size_t n = (size_t)h->g.n;
    mdk::KArgs a = h->a;
    a.snap = c->pool + 3 * n * (size_t)slot;
    a.snap_species = c->species;
    int rc;
    if ((rc = launch(h, h->ks->snapshot, h->g.nblk_i, kIntBlock, a)))
        return rc;
    int64_t spacing = 1;
    for (int b = 0; b < c->k; ++b, spacing *= c->l) {
        if (c->m % spacing)
            break;
        std::vector<int> &blk = c->blocks[b];
        blk.push_back(slot);
        c->refs[slot] += 1;
        if ((int)blk.size() < c->l)
            continue;
        mdk::CorrArgs ca;
        ca.s0 = c->pool + 3 * n * (size_t)blk[0];
        for (int j = 1; j < c->l; ++j)
            ca.sj[j - 1] = c->pool + 3 * n * (size_t)blk[j];
        for (int j = c->l; j <= mdk::kCorrMaxJ; ++j)
            ca.sj[j - 1] = nullptr;
        ca.nj = c->l - 1;
        ca.n = (int)n;
        ca.nq = c->nq;
        ca.species = c->species;
        ca.q = c->q;
        ca.part = c->part;
        ca.acc = c->acc + (size_t)b * (c->l - 1) * 4;
        ca.nblocks = c->nblocks;
        mdk::k_corr<<<c->nblocks, mdk::kCorrBlock, 0, h->s>>>(ca);
        mdk::k_corr_reduce<<<1, 128, 0, h->s>>>(ca);
        CK(h, cudaGetLastError());
        for (int j = 0; j < c->l - 1; ++j)
            c->origins[(size_t)b * (c->l - 1) + j] += 1;
        c->refs[blk[0]] -= 1;
        blk.erase(blk.begin());
    }
    c->m += 1;
    return MD_OK;
}

int md_corr_result(md_corr *c, int64_t *lags, double *msd, double *fs, int64_t *origins)
{
    ApiRange range_("md_corr_result");
    if (!c)
        return MD_E_INVAL;
    md_handle *h = c->h;
    const size_t nl = (size_t)c->k * (c->l - 1);
    std::vector<double> acc(4 * nl);
    CK(h, cudaStreamSynchronize(h->s));
    CK(h, cudaMemcpy(acc.data(), c->acc, sizeof(double) * 4 * nl, cudaMemcpyDeviceToHost));
    int64_t spacing = 1;
    for (int b = 0; b < c->k; ++b, spacing *= c->l)
        for (int j = 1; j < c->l; ++j) {
            const size_t t = (size_t)b * (c->l - 1) + (j - 1);
            const int64_t no = c->origins[t];
            if (lags)
                lags[t] = (int64_t)j * spacing;
            if (origins)
                origins[t] = no;
            for (int a = 0; a < 2; ++a) {
                const double cnt = (double)no * (double)h->n_species[a];
                const double nan = std::nan("");
                if (msd)
                    msd[2 * t + a] = cnt > 0 ? acc[4 * t + 2 * a] / cnt : nan;
                if (fs)
                    fs[2 * t + a] = cnt > 0 ? acc[4 * t + 2 * a + 1] / cnt : nan;
            }
        }
    return MD_OK;
}

int md_corr_destroy(md_corr *c)
{
    delete c;
    return MD_OK;
}

int md_compute_forces(md_handle *h, double *f, double *e, md_obs *totals)
{
    ApiRange range_("md_compute_forces");
    if (!h)
        return MD_E_INVAL;
    int rc;
    const size_t n = (size_t)h->g.n;
    if ((rc = launch(h, h->ks->mark_rebuild, 1, 1, h->a)) || (rc = launch_rebuild(h)) ||
        (rc = launch_force(h, 1)) || (rc = launch_integrate(h, mdk::IM_TOTALS)) ||
        (rc = launch(h, h->ks->expforce, grid_n(h->g.n, kIntBlock), kIntBlock, h->a)))
        return rc;
    if ((rc = check_device(h)))
        return rc;
    const size_t tb = sizeof(md_obs) * h->g.R;
    if ((rc = ensure_pinned(h, 32 * n + tb + 512)))
        return rc;
    char *q = h->pin;
    CK(h, cudaMemcpyAsync(q, h->a.st_f, 24 * n, cudaMemcpyDeviceToHost, h->s));
    CK(h, cudaMemcpyAsync(q + 24 * n, h->a.st_e, 8 * n, cudaMemcpyDeviceToHost, h->s));
    CK(h, cudaMemcpyAsync(q + 32 * n, h->a.totals, tb, cudaMemcpyDeviceToHost, h->s));
    CK(h, cudaStreamSynchronize(h->s));
    if (f)
        memcpy(f, q, 24 * n);
    if (e)
        memcpy(e, q + 24 * n, 8 * n);
    if (totals)
        memcpy(totals, q + 32 * n, tb);
    return MD_OK;
}

int md_observables(md_handle *h, md_obs *out, int32_t max_samples, int32_t *n_samples)
{
    ApiRange range_("md_observables");
    if (!h || !n_samples || (max_samples > 0 && !out))
        return MD_E_INVAL;
    *n_samples = 0;
    mdk::Ctl c;
    int rc = read_ctl(h, &c);
    if (rc)
        return rc;
    const int64_t avail = c.obs_count - h->obs_read;
    int64_t m = std::min<int64_t>(avail, h->cap);
    m = std::min<int64_t>(m, max_samples);
    const int64_t first = c.obs_count - m;
    const size_t rec = sizeof(md_obs) * h->g.R;
    if (m > 0) {
        if ((rc = ensure_pinned(h, rec * (size_t)m)))
            return rc;
        int64_t done = 0;
        while (done < m) {
            const int64_t slot = (first + done) % h->cap;
            const int64_t cnt = std::min<int64_t>(m - done, h->cap - slot);
            CK(h, cudaMemcpyAsync(h->pin + rec * done, (char *)h->a.ring + rec * slot, rec * cnt,
                                  cudaMemcpyDeviceToHost, h->s));
            done += cnt;
        }
        CK(h, cudaStreamSynchronize(h->s));
        memcpy(out, h->pin, rec * (size_t)m);
    }
    h->obs_read = c.obs_count;
    *n_samples = (int32_t)m;
    const int code = status_code(c.status);
    if (code != MD_OK)
        return check_device(h);
    return MD_OK;
}

int md_epot_series(md_handle *h, int64_t *steps, double *e_pot, int32_t max_steps, int32_t *n_steps)
{
    ApiRange range_("md_epot_series");
    if (!h || !n_steps || (max_steps > 0 && (!steps || !e_pot)))
        return MD_E_INVAL;
    *n_steps = 0;
    int rc = flush_epot(h);
    if (rc)
        return rc;
    mdk::Ctl c;
    if ((rc = read_ctl(h, &c)))
        return rc;
    const size_t cap = (size_t)h->cap, R = (size_t)h->g.R;
    const size_t sb = align_up(sizeof(long long) * cap);
    if ((rc = ensure_pinned(h, sb + sizeof(double) * cap * R)) || (rc = stage_wait(h)))
        return rc;
    CK(h, cudaMemcpyAsync(h->pin, h->a.epot_step, sizeof(long long) * cap, cudaMemcpyDeviceToHost, h->s));
    CK(h, cudaMemcpyAsync(h->pin + sb, h->a.epot, sizeof(double) * cap * R, cudaMemcpyDeviceToHost, h->s));
    CK(h, cudaStreamSynchronize(h->s));
    const long long *st = (const long long *)h->pin;
    const double *ev = (const double *)(h->pin + sb);
    std::vector<std::pair<long long, size_t>> got;       // (step, slot) not yet returned
    for (size_t k = 0; k < cap; ++k)
        if (st[k] > h->epot_read)
            got.push_back({st[k], k});
    std::sort(got.begin(), got.end());
    const size_t m = std::min<size_t>(got.size(), (size_t)std::max(max_steps, 0));
    const size_t first = got.size() - m;                  // the newest m
    for (size_t t = 0; t < m; ++t) {
        steps[t] = got[first + t].first;
        memcpy(e_pot + t * R, ev + got[first + t].second * R, sizeof(double) * R);
    }
    if (!got.empty())
        h->epot_read = got.back().first;
    *n_steps = (int32_t)m;
    if (status_code(c.status) != MD_OK)
        return check_device(h);
    return MD_OK;
}

int md_get_state(md_handle *h, double *pos, double *vel, int32_t *image)
{
    ApiRange range_("md_get_state");
    if (!h)
        return MD_E_INVAL;
    int rc;
    const size_t n = (size_t)h->g.n;
    if ((rc = launch(h, h->ks->getstate, grid_n(h->g.n, kIntBlock), kIntBlock, h->a)))
        return rc;
    if ((rc = ensure_pinned(h, 60 * n)) || (rc = stage_wait(h)))
        return rc;
    char *q = h->pin;
    CK(h, cudaMemcpyAsync(q, h->a.st_pos, 24 * n, cudaMemcpyDeviceToHost, h->s));
    CK(h, cudaMemcpyAsync(q + 24 * n, h->a.st_vel, 24 * n, cudaMemcpyDeviceToHost, h->s));
    CK(h, cudaMemcpyAsync(q + 48 * n, h->a.st_img, 12 * n, cudaMemcpyDeviceToHost, h->s));
    CK(h, cudaStreamSynchronize(h->s));
    if (pos)
        memcpy(pos, q, 24 * n);
    if (vel)
        memcpy(vel, q + 24 * n, 24 * n);
    if (image)
        memcpy(image, q + 48 * n, 12 * n);
    return MD_OK;
}

int md_set_state(md_handle *h, const double *pos, const double *vel, const int32_t *image)
{
    ApiRange range_("md_set_state");
    if (!h || !pos || !vel)
        return MD_E_INVAL;
    int rc;
    // species are kept: read them back from the working layout is not needed,
    // the staging area still holds the codes uploaded at creation
    const size_t n = (size_t)h->g.n;
    if ((rc = ensure_pinned(h, 64 * n)) || (rc = stage_wait(h)))
        return rc;
    char *q = h->pin;
    memcpy(q, pos, 24 * n);
    memcpy(q + 24 * n, vel, 24 * n);
    if (image)
        memcpy(q + 48 * n, image, 12 * n);
    else
        memset(q + 48 * n, 0, 12 * n);
    CK(h, cudaMemcpyAsync(h->a.st_pos, q, 24 * n, cudaMemcpyHostToDevice, h->s));
    CK(h, cudaMemcpyAsync(h->a.st_vel, q + 24 * n, 24 * n, cudaMemcpyHostToDevice, h->s));
    CK(h, cudaMemcpyAsync(h->a.st_img, q + 48 * n, 12 * n, cudaMemcpyHostToDevice, h->s));
    CK(h, cudaEventRecord(h->ev_stage, h->s));
    if ((rc = launch(h, h->ks->load, h->g.nblk_i, kIntBlock, h->a)) || (rc = launch_rebuild(h)))
        return rc;
    return launch_force(h, 1);
}

int md_get_neighbours(md_handle *h, int32_t *counts, int32_t *lists, int32_t kmax)
{
    ApiRange range_("md_get_neighbours");
    if (!h || !counts || (lists && kmax < 1))
        return MD_E_INVAL;
    const size_t n = (size_t)h->g.n;
    int rc;
    mdk::Ctl c;
    if ((rc = read_ctl(h, &c)))
        return rc;
    const size_t K = (size_t)h->g.Kmax;                  // row stride of the lists (the cap)
    if ((rc = ensure_pinned(h, 4 * n * K + 4 * n + 16 * n + 256)) || (rc = stage_wait(h)))
        return rc;
    char *q = h->pin;
    int *nn = (int *)q;
    int4 *img = (int4 *)(q + align_up(4 * n));
    int *nb = (int *)(q + align_up(4 * n) + align_up(16 * n));
    const int4 *dimg = c.state_par ? h->a.image2 : h->a.image;   // tags of the current order
    CK(h, cudaMemcpyAsync(nn, h->a.nnbr, 4 * n, cudaMemcpyDeviceToHost, h->s));
    CK(h, cudaMemcpyAsync(img, dimg, 16 * n, cudaMemcpyDeviceToHost, h->s));
    if (lists)
        CK(h, cudaMemcpyAsync(nb, h->a.nbr, 4 * n * K, cudaMemcpyDeviceToHost, h->s));
    CK(h, cudaStreamSynchronize(h->s));
    for (size_t s = 0; s < n; ++s) {
        const int t = img[s].w;
        counts[t] = nn[s];
        if (lists) {
            for (int k = 0; k < kmax; ++k)
                lists[(size_t)t * kmax + k] = (k < nn[s] && (size_t)k < K) ? img[nb[s * K + k]].w : -1;
        }
    }
    return MD_OK;
}

int md_info(md_handle *h, md_info_t *out)
{
    if (!h || !out)
        return MD_E_INVAL;
    mdk::Ctl c;
    int rc = read_ctl(h, &c);
    if (rc)
        return rc;
    memset(out, 0, sizeof *out);
    out->n_total = h->g.n;
    out->n_replicas = h->g.R;
    out->neigh_capacity = c.K;
    out->neigh_capacity_max = h->g.Kmax;
    out->regrows = c.regrows;
    out->build_form = h->g.nb_block ? 2 : 1;
    out->step_form = h->g.sweep ? 2 : 1;
    out->threads_per_particle = h->g.tpp;
    out->check_interval = h->g.check;
    out->cells_per_edge = h->g.rep[0].nc;
    out->step = c.step;
    out->rebuilds = c.rebuilds;
    out->kernel_launches = c.n_force + c.n_integrate + c.n_rebuild_k + c.n_other;
    out->max_neighbours = c.max_nbr;
    out->status = status_code(c.status);
    out->step_ms = h->step_ms;
    out->step_launches = h->step_launches;
    out->rebuild_ms = h->rebuild_ms;
    out->rebuild_checks = h->rebuild_checks;
    out->step_device_ms = (double)c.dev_ns * 1e-6;
    out->step_device_launches = c.dev_launches;
    return MD_OK;
}

int md_sync(md_handle *h)
{
    if (!h)
        return MD_E_INVAL;
    return check_device(h);
}

int md_destroy(md_handle *h)
{
    ApiRange range_("md_destroy");
    if (!h)
        return MD_E_INVAL;
    if (h->ws)
        cudaStreamSynchronize(h->s);
    if (h->gexec)
        cudaGraphExecDestroy(h->gexec);
    if (h->graph)
        cudaGraphDestroy(h->graph);
    if (h->pin)
        cudaFreeHost(h->pin);
    if (h->ev_stage)
        cudaEventDestroy(h->ev_stage);
    if (h->ev_f0)
        cudaEventDestroy(h->ev_f0);
    if (h->ev_f1)
        cudaEventDestroy(h->ev_f1);
    if (h->ev_i1)
        cudaEventDestroy(h->ev_i1);
    delete h;
    return MD_OK;
}

const char *md_last_error(const md_handle *h)
{
    if (!h)
        return md_noalloc_message();
    return h->err.c_str();
}

const char *md_status_string(int code)
{
    switch (code) {
    case MD_OK: return "MD_OK";
    case MD_E_INVAL: return "MD_E_INVAL";
    case MD_E_NOMEM: return "MD_E_NOMEM";
    case MD_E_CUDA: return "MD_E_CUDA";
    case MD_E_NONFINITE: return "MD_E_NONFINITE";
    case MD_E_UNSTABLE: return "MD_E_UNSTABLE";
    case MD_E_TIMEOUT: return "MD_E_TIMEOUT";
    case MD_E_CAPACITY: return "MD_E_CAPACITY";
    case MD_E_BOUNDS: return "MD_E_BOUNDS";
    default: return "MD_E_UNKNOWN";
    }
}

}  // extern "C"
