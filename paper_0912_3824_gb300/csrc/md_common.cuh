// md_common.cuh -- device-side data structures and double-single arithmetic
// shared by the kernels and the host API of the GB300 MD library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mdk {

// precision modes (same values as MD_PREC_* in md.h)
enum { FP64 = 0, MIXED = 1, FP32 = 2 };

// device status bits
enum { ST_OVERFLOW = 1u, ST_NONFINITE = 2u, ST_UNSTABLE = 4u, ST_TIMEOUT = 8u, ST_BOUNDS = 16u };

// integrate-kernel modes
enum {
    IM_FIRST = 0,   // half kick + drift (start of md_step)
    IM_LOOP = 1,    // half kick, sample, then half kick + drift unless this is the last step
    IM_SAMPLE = 2,  // kinetic reductions only; record a ring-buffer sample
    IM_TOTALS = 3,  // kinetic reductions only; write the per-replica totals record
    IM_KE = 4       // kinetic energy only; turn targets in scale[] into rescale factors
};

// neighbour-list radius margin and rebuild-threshold margin (absolute, sigma units):
// they absorb the single-precision rounding of distances and displacements.
constexpr float kListMargin = 1e-4f;
constexpr float kDispMargin = 1e-4f;

// Control block in device memory, written by the kernels.
struct Ctl {
    unsigned int status;      // ST_* bits
    unsigned int rebuild;     // 1: lists must be rebuilt before the next force evaluation
    unsigned int maxdisp2;    // float bits of the largest squared displacement (this step)
    unsigned int ticket;      // last-block counter of the step / integrate kernels
    unsigned int maxv2;       // float bits of the largest squared speed (this step)
    unsigned int maxa2;       // float bits of the largest squared acceleration (this step)
    int pos_par;              // which of the two position buffers is current
    int state_par;            // which of the two velocity / image buffers is current
    int max_nbr;              // largest list length seen at the last build
    int K;                    // list entries per particle in use; grows on the device when a
                              // build finds a longer list, up to Kmax
    int Kmax;                 // capacity cap: the row stride of nbr (KArgs::Kstride)
    unsigned int regrow;      // 1: the last build overflowed K; K was raised and the build
                              // must be redone before the lists are used
    long long step;           // time index of the current positions
    long long remaining;      // force evaluations left in the running md_step
    long long budget;         // loop-iteration bound of the running md_step
    long long rebuilds;
    long long obs_count;      // samples written to the ring
    long long n_force, n_integrate, n_rebuild_k, n_other;   // kernel executions
    unsigned long long t_first_inv;   // step kernel: ~(earliest block start, %globaltimer ns) of the
                                      // running launch (0 = none yet; atomicMax of the complement)
    unsigned long long dev_ns;        // summed device duration of the step-kernel launches
    long long dev_launches;
    float last_maxdisp2;
    float pad1;
    long long regrows;        // builds redone with a larger K since md_create
    long long epot_pending;   // a step whose warp energy partials still await their sum (-1: none)
};

struct Rep {                  // one independent system
    int start, n;             // particle range (sorted order keeps replicas contiguous)
    int cell0, nc;            // first global cell id, cells per edge (1 if fewer than 3 fit)
    int bi0, bi1;             // integrate-kernel block range
    int bf0, bf1;             // force-kernel block range
    double L, invL, cscale;   // box edge, 1/L, nc/L
    float Lhi, Llo, invLf, cscalef;
    float grid, inv_grid;     // anchoring grid of MIXED positions (powers of two)
    float qunit;              // L / 2^32: length of one unit of the fixed-point positions
    float qscale;             // 2^32 / L (single precision): units per length
    unsigned long long qgrid; // grid * 2^32 / L in units of 2^-28: units per grid step, fixed point
    double mtot;              // total mass of the replica
};

struct PairTab {              // [a*2+b]
    float rc2[4], rl2[4], sig2[4], eps4[4], eps48[4], shift[4];
    float rc[4], ihs[4];      // r_c and 1 / (h sigma) of the smoothing (Sec. 4)
    float vc[4];              // S_ab / (4 eps_ab) (0 where eps_ab = 0): V = 4 eps_ab (s6^2 - s6 - vc)
    double rc2d[4], rl2d[4], sig2d[4], eps4d[4], eps48d[4], shiftd[4];
    double rcd[4], ihsd[4], vcd[4];
};

struct Obs {                  // identical layout to md_obs
    long long step;
    double e_pot, e_kin, virial, w[6], p[3], max_disp;
    long long rebuilds;
};

struct __align__(32) d4 { double x, y, z, w; };

// Every kernel takes this one struct by value.
struct KArgs {
    int n, nrep, ncell, tpp, si, obs_cap, epot_cap, imode, use_cond, fsample;
    int Kstride;                      // list row stride: the capacity cap (Ctl::Kmax); the rows hold
                                      // at most Ctl::K entries, so K can grow without a new layout
    int nblk_i, nblk_f;
    int lookahead;                    // MD steps until the next rebuild check (after this node)
    int set_rebuild, set_loop;        // this graph node sets the rebuild / loop condition
    int nb_retry;                     // neighbour build: 0 = first pass, 1 = the redo after a regrow
    int set_regrow;                   // this build node sets the regrow condition
    void *pa, *pb, *va, *vb;          // buffer 0: MIXED pos hi/lo, vel hi/lo (float4);
                                      // FP64 pos, vel (d4); FP32 pos, vel (float4)
    void *pa2, *pb2, *va2, *vb2;      // buffer 1 (positions: Ctl::pos_par, velocities: state_par)
    int4 *qa, *qb;                    // MIXED: fixed-point copy of the positions (x/L in units of
                                      // 2^-32, species in w) read by the pair loops; by Ctl::pos_par
    void *force;                      // float4 (MIXED, FP32) or d4 (FP64): f.xyz, e_i in w
    float4 *rref;                     // positions at the last list build
    int4 *image, *image2;             // image counters (w = original index), by state_par
    int *key, *ccount, *cstart, *ccursor, *tmpidx;
    int *skey;                        // sub-cell code of each particle (order inside its cell)
    const int *crank;                 // [global linear cell] -> global sorted cell id
    const int4 *cxyz;                 // [global sorted cell id] -> cx, cy, cz, replica
    int *nbr, *nnbr;
    const int4 *blk_i, *blk_f;        // per block: first particle, end, replica (blk_f: + its
                                      // chunk index, the slot of its partial sums)
    const int4 *blk_s;                // step kernel: rows of blk_f in the order the resident blocks
                                      // take them, cpb per block (w = -1: padding)
    int cpb;                          // step kernel: chunks per block
    double *part_f, *part_i;          // per-block partial sums [nblk_f][12], [nblk_i][4]
    void *part_e;                     // per-block potential energy [nblk_f]: double (FP64 mode) or
                                      // float2 double-single (MIXED, FP32)
    Obs *ring, *totals;
    double *epot;                     // per-step potential energy [epot_cap][nrep], slot = step % cap
    long long *epot_step;             // [epot_cap]: the step held by each slot (-1 = none)
    Ctl *ctl;
    const Rep *rep;
    double *st_pos, *st_vel, *st_f, *st_e;   // staging, original order
    int *st_img, *st_code;
    double *scale;                    // [nrep] targets in, factors out (rescale)
    unsigned long long r48_x0;        // Andersen heat bath (Sec. 2.3): rand48 state after seeding,
    unsigned long long r48_AN, r48_CN;//   leapfrog multiplier / addend over n threads,
    long long r48_base;               //   first deviate index of the collision (4 * event * n)
    double *snap;                     // time-correlation snapshot: unwrapped positions [n][3] and
    int *snap_species;                //   species, both by original particle index
    PairTab tab;
    double hdtm[2], dt, mass[2];      // dt / (2 m_a), dt, m_a
    long long nsteps;                 // for k_set_steps
    float hdtm_hi[2], hdtm_lo[2], dt_hi, dt_lo, inv_mass[2];
    float disp_thr2, disp_thr;        // (skin/2 - margin)^2 and skin/2 - margin
    long long budget;                 // for k_set_steps: step-loop bound (0 = nsteps + 64)
    cudaGraphConditionalHandle h_loop, h_rebuild, h_regrow;
};

// ---------------------------------------------------------------------------
// Double-single arithmetic (Sec. 2.4, Algorithm 1): a value is hi + lo with
// |lo| <= ulp(hi)/2.  Sums use Knuth's branch-free two-sum, products the
// exact fmaf residual; the intrinsics keep the compiler from contracting or
// reassociating the error terms.
// ---------------------------------------------------------------------------
struct ds { float hi, lo; };

__device__ __forceinline__ ds ds_from(float hi, float lo) { ds r; r.hi = hi; r.lo = lo; return r; }

// renormalise s + e with |e| small against s (Dekker's fast two-sum)
__device__ __forceinline__ ds ds_norm(float s, float e)
{
    float h = __fadd_rn(s, e);
    return ds_from(h, __fsub_rn(e, __fsub_rn(h, s)));
}

// a + b, both double-single
__device__ __forceinline__ ds ds_add(ds a, ds b)
{
    float s = __fadd_rn(a.hi, b.hi);
    float bb = __fsub_rn(s, a.hi);                       // part of s that came from b
    float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    err = __fadd_rn(__fadd_rn(err, a.lo), b.lo);
    return ds_norm(s, err);
}

// a * b for double-single a and single b
__device__ __forceinline__ ds ds_mul_f(ds a, float b)
{
    float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);                    // exact rounding error of a.hi*b
    e = __fmaf_rn(a.lo, b, e);
    return ds_norm(p, e);
}

// a * b, both double-single
__device__ __forceinline__ ds ds_mul(ds a, ds b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ds_norm(p, e);
}

__device__ __forceinline__ double ds_to_double(ds a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ ds ds_from_double(double x)
{
    float hi = __double2float_rn(x);
    return ds_from(hi, __double2float_rn(x - (double)hi));
}

// table of kernel entry addresses for one precision (one translation unit each)
struct KernelSet {
    const void *integrate, *force[2][6], *step[2][6];   // [smoothed][log2 lanes per particle]
    const void *step_sweep[2][2];     // step kernel, resident blocks sweeping runs of chunks
                                      // (single-precision pair loops, 1 or 2 lanes; else null)
    const void *bin, *scan, *scatter, *permute, *nbuild, *nbuild_blk;
    const void *load, *getstate, *expforce, *scale, *set_steps, *reset, *mark_rebuild;
    const void *andersen, *andersen_fix, *snapshot, *epot_flush;
};

const KernelSet &kernels_fp64();
const KernelSet &kernels_mixed();
const KernelSet &kernels_fp32();

}  // namespace mdk
