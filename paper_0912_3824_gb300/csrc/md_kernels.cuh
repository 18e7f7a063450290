// md_kernels.cuh -- the MD step kernels, templated on the precision mode.
//
// Included by one translation unit per precision (md_kernels_{fp64,mixed,fp32}.cu),
// each of which instantiates every kernel for its mode and exports a table of
// kernel entry addresses.  All kernels take one KArgs by value.
//
// State layout in device memory (slot order = cell order after each rebuild):
//   MIXED  pa: float4 (H.x, H.y, H.z, species bits)  pb: float4 (l.x, l.y, l.z, 0)
//          position = H + l, H on a power-of-two grid of the box (see anchor())
//          va / vb: float4 velocity high / low words (normalised double-single)
//   FP64   pa: d4 (x, y, z, species bits), va: d4 velocity
//   FP32   pa: float4 (x, y, z, species bits), va: float4 velocity
//   force: float4 (MIXED, FP32) or d4 (FP64): (Fx, Fy, Fz, e_i)
//   image: int4 (nx, ny, nz, original index)
#pragma once

#include "md_common.cuh"

namespace mdk {

constexpr int kIntBlock = 256;   // per-particle kernels: one thread per particle
constexpr int kForceBlock = 256; // force kernel: tpp threads per particle
constexpr int kNbBlock = 256;    // neighbour build: one warp per particle
constexpr int kScanBlock = 1024;

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum NV doubles over the block in a fixed order; thread 0 ends with the sums.
// sh: shared scratch of 32*NV doubles.  Every thread of the block must call it.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        v[k] = warp_sum(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k)
            sh[w * NV + k] = v[k];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = lane < nw ? sh[lane * NV + k] : 0.0;
            v[k] = warp_sum(x);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ float block_max(float v, float *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_max(v);
    if (lane == 0)
        sh[w] = v;
    __syncthreads();
    if (w == 0) {
        float x = lane < nw ? sh[lane] : 0.0f;
        v = warp_max(x);
    }
    __syncthreads();
    return v;
}

__device__ __forceinline__ int species_of(float w) { return __float_as_int(w) & 15; }
__device__ __forceinline__ int species_of(double w) { return (int)(__double_as_longlong(w) & 15); }

// Re-anchor a double-single coordinate so that its high word lies on the grid
// of spacing `grid` (a power of two chosen so that every coordinate in
// [-L, 2L) is exactly representable on it), then wrap it into [0, L).
// Differences of anchored high words, and their shift by the anchored box
// edge Lhi, are exact in single precision; this is what makes the
// single-precision pair separation accurate for pairs across the boundary.
// Returns the change of the image counter (-1, 0, 1).
__device__ __forceinline__ int anchor_wrap(ds x, float grid, float inv_grid, float Lhi, float Llo,
                                           float &H, float &l)
{
    float h = __fmul_rn(rintf(__fmul_rn(x.hi, inv_grid)), grid);  // power-of-two scalings: exact
    float r = __fadd_rn(__fsub_rn(x.hi, h), x.lo);                 // x.hi - h is exact
    int img = 0;
    if (h > Lhi || (h == Lhi && r >= Llo)) {
        h = __fsub_rn(h, Lhi);
        r = __fsub_rn(r, Llo);
        img = 1;
    } else if (h < 0.0f || (h == 0.0f && r < 0.0f)) {
        h = __fadd_rn(h, Lhi);
        r = __fadd_rn(r, Llo);
        img = -1;
    }
    H = h;
    l = r;
    return img;
}

// Minimum-image separation component from anchored double-single coordinates.
// d = Hi - Hj and d - k*Lhi are exact; only the final sum rounds.
__device__ __forceinline__ float sep_ds(float Hi, float li, float Hj, float lj,
                                        float Lhi, float Llo, float invL)
{
    float d = __fsub_rn(Hi, Hj);
    float k = rintf(__fmul_rn(d, invL));
    float dh = __fmaf_rn(-k, Lhi, d);
    float dl = __fmaf_rn(-k, Llo, __fsub_rn(li, lj));
    return __fadd_rn(dh, dl);
}

__device__ __forceinline__ float sep_f(float xi, float xj, float L, float invL)
{
    float d = xi - xj;
    return fmaf(-rintf(d * invL), L, d);
}

__device__ __forceinline__ double sep_d(double xi, double xj, double L, double invL)
{
    double d = xi - xj;
    return fma(-rint(d * invL), L, d);
}

// Kahan-compensated accumulation: the running sum is s - c.
__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    float y = __fsub_rn(x, c);
    float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// ---------------------------------------------------------------------------
// state access
// ---------------------------------------------------------------------------
template <int P> struct Vec;
template <> struct Vec<MIXED> { ds x, y, z; };
template <> struct Vec<FP64> { double x, y, z; };
template <> struct Vec<FP32> { float x, y, z; };

// ---------------------------------------------------------------------------
// integrate: velocity-Verlet half kicks and drift (Sec. 2.2), the per-step
// maximum-displacement reduction that decides the list rebuild, and the
// kinetic reductions; its last block finishes all reductions, advances the
// step counter and sets the graph conditions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void write_record(const KArgs &a, int r, const double *v, long long step,
                                             float md2, long long rebuilds, long long slot)
{
    Obs o;
    o.step = step;
    o.e_pot = v[0];
    o.virial = v[1];
    for (int k = 0; k < 6; ++k)
        o.w[k] = v[2 + k];
    o.e_kin = v[8];
    o.p[0] = v[9];
    o.p[1] = v[10];
    o.p[2] = v[11];
    o.max_disp = sqrt((double)md2);
    o.rebuilds = rebuilds;
    if (a.imode == IM_TOTALS)
        a.totals[r] = o;
    else if (a.imode == IM_KE) {
        const Rep &rp = a.rep[r];
        double dof = 3.0 * (double)rp.n - 3.0;
        double target = a.scale[r];
        a.scale[r] = (v[8] > 0.0) ? sqrt(target * dof / (2.0 * v[8])) : 1.0;
    } else
        a.ring[slot * a.nrep + r] = o;
}

// Per-replica reduction of the force-kernel and integrate-kernel block partials,
// in a fixed order (deterministic).  Runs in the last block of k_integrate.
static __device__ void finish_reductions(const KArgs &a, long long step, float md2, double *sh)
{
    const Ctl *ctl = a.ctl;
    const long long slot = ctl->obs_count % (long long)a.obs_cap;
    const long long rebuilds = ctl->rebuilds;
    const bool want_f = a.imode != IM_KE;
    if (a.nrep <= 8) {
        for (int r = 0; r < a.nrep; ++r) {
            const Rep rp = a.rep[r];
            double v[12];
#pragma unroll
            for (int k = 0; k < 12; ++k)
                v[k] = 0.0;
            if (want_f)
                for (int b = rp.bf0 + threadIdx.x; b < rp.bf1; b += blockDim.x)
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        v[k] += a.part_f[(size_t)b * 8 + k];
            for (int b = rp.bi0 + threadIdx.x; b < rp.bi1; b += blockDim.x)
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    v[8 + k] += a.part_i[(size_t)b * 4 + k];
            block_sum<12>(v, sh);
            if (threadIdx.x == 0)
                write_record(a, r, v, step, md2, rebuilds, slot);
        }
    } else {
        for (int r = threadIdx.x; r < a.nrep; r += blockDim.x) {
            const Rep rp = a.rep[r];
            double v[12];
            for (int k = 0; k < 12; ++k)
                v[k] = 0.0;
            if (want_f)
                for (int b = rp.bf0; b < rp.bf1; ++b)
                    for (int k = 0; k < 8; ++k)
                        v[k] += a.part_f[(size_t)b * 8 + k];
            for (int b = rp.bi0; b < rp.bi1; ++b)
                for (int k = 0; k < 4; ++k)
                    v[8 + k] += a.part_i[(size_t)b * 4 + k];
            write_record(a, r, v, step, md2, rebuilds, slot);
        }
        __syncthreads();
    }
}

template <int P>
__global__ void __launch_bounds__(kIntBlock) k_integrate(KArgs a)
{
    __shared__ double sh[32 * 12];
    __shared__ float shf[32];
    __shared__ int s_last;
    __shared__ float s_md2;
    Ctl *ctl = a.ctl;

    const unsigned int st0 = ctl->status;
    const bool halted = st0 != 0u;
    const long long step = ctl->step;
    const long long remaining = ctl->remaining;
    const int mode = a.imode;
    const bool kickA = (mode == IM_LOOP);                              // completes v(t)
    const bool last = (mode == IM_LOOP) && remaining <= 1;
    const bool kickB = (mode == IM_FIRST) || (mode == IM_LOOP && !last); // starts step t+1
    const bool rec = (mode == IM_LOOP && (step % a.si) == 0) || mode == IM_SAMPLE ||
                     mode == IM_TOTALS || mode == IM_KE;

    const int4 b = a.blk_i[blockIdx.x];
    const Rep rp = a.rep[b.z];
    const int i = b.x + threadIdx.x;
    const bool valid = (i < b.y) && !halted;

    float disp2 = 0.0f;
    double kin[4] = {0.0, 0.0, 0.0, 0.0};
    unsigned int bad = 0u;

    if (valid) {
        if constexpr (P == MIXED) {
            float4 H = ((float4 *)a.pa)[i], l = ((float4 *)a.pb)[i];
            float4 vh = ((float4 *)a.va)[i], vl = ((float4 *)a.vb)[i];
            const int sp = species_of(H.w);
            Vec<MIXED> v{ds_from(vh.x, vl.x), ds_from(vh.y, vl.y), ds_from(vh.z, vl.z)};
            const ds hk = ds_from(a.hdtm_hi[sp], a.hdtm_lo[sp]);
            float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kickA || kickB)
                f = ((const float4 *)a.force)[i];
            if (kickA) {
                v.x = ds_add(v.x, ds_mul_f(hk, f.x));
                v.y = ds_add(v.y, ds_mul_f(hk, f.y));
                v.z = ds_add(v.z, ds_mul_f(hk, f.z));
            }
            if (rec) {
                const double m = a.mass[sp];
                double dx = ds_to_double(v.x), dy = ds_to_double(v.y), dz = ds_to_double(v.z);
                kin[0] = 0.5 * m * (dx * dx + dy * dy + dz * dz);
                kin[1] = m * dx;
                kin[2] = m * dy;
                kin[3] = m * dz;
            }
            if (kickB) {
                v.x = ds_add(v.x, ds_mul_f(hk, f.x));
                v.y = ds_add(v.y, ds_mul_f(hk, f.y));
                v.z = ds_add(v.z, ds_mul_f(hk, f.z));
                const ds dt = ds_from(a.dt_hi, a.dt_lo);
                ds sx = ds_mul(dt, v.x), sy = ds_mul(dt, v.y), sz = ds_mul(dt, v.z);
                const float lim = 0.25f * rp.Lhi;
                if (fabsf(sx.hi) > lim || fabsf(sy.hi) > lim || fabsf(sz.hi) > lim)
                    bad |= ST_UNSTABLE;
                ds nx = ds_add(ds_from(H.x, l.x), sx);
                ds ny = ds_add(ds_from(H.y, l.y), sy);
                ds nz = ds_add(ds_from(H.z, l.z), sz);
                int ix = anchor_wrap(nx, rp.grid, rp.inv_grid, rp.Lhi, rp.Llo, H.x, l.x);
                int iy = anchor_wrap(ny, rp.grid, rp.inv_grid, rp.Lhi, rp.Llo, H.y, l.y);
                int iz = anchor_wrap(nz, rp.grid, rp.inv_grid, rp.Lhi, rp.Llo, H.z, l.z);
                if (!isfinite(H.x) || !isfinite(H.y) || !isfinite(H.z))
                    bad |= ST_NONFINITE;
                if (ix | iy | iz) {
                    int4 im = a.image[i];
                    im.x += ix;
                    im.y += iy;
                    im.z += iz;
                    a.image[i] = im;
                }
                ((float4 *)a.pa)[i] = H;
                ((float4 *)a.pb)[i] = l;
                const float4 rr = a.rref[i];
                float ddx = __fadd_rn(sep_f(H.x, rr.x, rp.Lhi, rp.invLf), l.x);
                float ddy = __fadd_rn(sep_f(H.y, rr.y, rp.Lhi, rp.invLf), l.y);
                float ddz = __fadd_rn(sep_f(H.z, rr.z, rp.Lhi, rp.invLf), l.z);
                disp2 = ddx * ddx + ddy * ddy + ddz * ddz;
            }
            if (kickA || kickB) {
                ((float4 *)a.va)[i] = make_float4(v.x.hi, v.y.hi, v.z.hi, 0.f);
                ((float4 *)a.vb)[i] = make_float4(v.x.lo, v.y.lo, v.z.lo, 0.f);
            }
        } else if constexpr (P == FP64) {
            d4 x = ((d4 *)a.pa)[i], v = ((d4 *)a.va)[i];
            const int sp = species_of(x.w);
            const double hk = a.hdtm[sp];
            d4 f = {0.0, 0.0, 0.0, 0.0};
            if (kickA || kickB)
                f = ((const d4 *)a.force)[i];
            if (kickA) {
                v.x += hk * f.x;
                v.y += hk * f.y;
                v.z += hk * f.z;
            }
            if (rec) {
                const double m = a.mass[sp];
                kin[0] = 0.5 * m * (v.x * v.x + v.y * v.y + v.z * v.z);
                kin[1] = m * v.x;
                kin[2] = m * v.y;
                kin[3] = m * v.z;
            }
            if (kickB) {
                v.x += hk * f.x;
                v.y += hk * f.y;
                v.z += hk * f.z;
                double sx = a.dt * v.x, sy = a.dt * v.y, sz = a.dt * v.z;
                const double lim = 0.25 * rp.L;
                if (fabs(sx) > lim || fabs(sy) > lim || fabs(sz) > lim)
                    bad |= ST_UNSTABLE;
                x.x += sx;
                x.y += sy;
                x.z += sz;
                int ix = 0, iy = 0, iz = 0;
                if (x.x >= rp.L) { x.x -= rp.L; ix = 1; } else if (x.x < 0.0) { x.x += rp.L; ix = -1; }
                if (x.y >= rp.L) { x.y -= rp.L; iy = 1; } else if (x.y < 0.0) { x.y += rp.L; iy = -1; }
                if (x.z >= rp.L) { x.z -= rp.L; iz = 1; } else if (x.z < 0.0) { x.z += rp.L; iz = -1; }
                if (!isfinite(x.x) || !isfinite(x.y) || !isfinite(x.z))
                    bad |= ST_NONFINITE;
                if (ix | iy | iz) {
                    int4 im = a.image[i];
                    im.x += ix;
                    im.y += iy;
                    im.z += iz;
                    a.image[i] = im;
                }
                ((d4 *)a.pa)[i] = x;
                const float4 rr = a.rref[i];
                float ddx = sep_f(__double2float_rn(x.x), rr.x, rp.Lhi, rp.invLf);
                float ddy = sep_f(__double2float_rn(x.y), rr.y, rp.Lhi, rp.invLf);
                float ddz = sep_f(__double2float_rn(x.z), rr.z, rp.Lhi, rp.invLf);
                disp2 = ddx * ddx + ddy * ddy + ddz * ddz;
            }
            if (kickA || kickB)
                ((d4 *)a.va)[i] = v;
        } else {  // FP32
            float4 x = ((float4 *)a.pa)[i], v = ((float4 *)a.va)[i];
            const int sp = species_of(x.w);
            const float hk = (float)a.hdtm[sp];
            float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kickA || kickB)
                f = ((const float4 *)a.force)[i];
            if (kickA) {
                v.x += hk * f.x;
                v.y += hk * f.y;
                v.z += hk * f.z;
            }
            if (rec) {
                const double m = a.mass[sp];
                double dx = v.x, dy = v.y, dz = v.z;
                kin[0] = 0.5 * m * (dx * dx + dy * dy + dz * dz);
                kin[1] = m * dx;
                kin[2] = m * dy;
                kin[3] = m * dz;
            }
            if (kickB) {
                v.x += hk * f.x;
                v.y += hk * f.y;
                v.z += hk * f.z;
                const float dt = (float)a.dt;
                float sx = dt * v.x, sy = dt * v.y, sz = dt * v.z;
                const float lim = 0.25f * rp.Lhi;
                if (fabsf(sx) > lim || fabsf(sy) > lim || fabsf(sz) > lim)
                    bad |= ST_UNSTABLE;
                x.x += sx;
                x.y += sy;
                x.z += sz;
                const float L = rp.Lhi;
                int ix = 0, iy = 0, iz = 0;
                if (x.x >= L) { x.x -= L; ix = 1; } else if (x.x < 0.f) { x.x += L; ix = -1; }
                if (x.y >= L) { x.y -= L; iy = 1; } else if (x.y < 0.f) { x.y += L; iy = -1; }
                if (x.z >= L) { x.z -= L; iz = 1; } else if (x.z < 0.f) { x.z += L; iz = -1; }
                if (x.x >= L) x.x = 0.f;   // x just below 0 can round to L when wrapped
                if (x.y >= L) x.y = 0.f;
                if (x.z >= L) x.z = 0.f;
                if (!isfinite(x.x) || !isfinite(x.y) || !isfinite(x.z))
                    bad |= ST_NONFINITE;
                if (ix | iy | iz) {
                    int4 im = a.image[i];
                    im.x += ix;
                    im.y += iy;
                    im.z += iz;
                    a.image[i] = im;
                }
                ((float4 *)a.pa)[i] = x;
                const float4 rr = a.rref[i];
                float ddx = sep_f(x.x, rr.x, L, rp.invLf);
                float ddy = sep_f(x.y, rr.y, L, rp.invLf);
                float ddz = sep_f(x.z, rr.z, L, rp.invLf);
                disp2 = ddx * ddx + ddy * ddy + ddz * ddz;
            }
            if (kickA || kickB)
                ((float4 *)a.va)[i] = v;
        }
    }
    if (bad)
        atomicOr(&ctl->status, bad);

    // block reductions
    const float bmax = block_max(disp2, shf);
    if (rec)
        block_sum<4>(kin, sh);
    if (threadIdx.x == 0) {
        if (rec) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                a.part_i[(size_t)blockIdx.x * 4 + k] = kin[k];
        }
        if (bmax > 0.0f)
            atomicMax(&ctl->maxdisp2, __float_as_uint(bmax));
        __threadfence();
        const unsigned int t = atomicAdd(&ctl->ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last)
        return;

    // ---- last block: all blocks' partials and flags are visible ----
    __threadfence();
    if (threadIdx.x == 0)
        s_md2 = __uint_as_float(atomicExch(&ctl->maxdisp2, 0u));
    __syncthreads();
    const unsigned int st = atomicOr(&ctl->status, 0u);
    const float md2 = s_md2;
    if (rec && st == 0u)
        finish_reductions(a, step, md2, sh);
    if (threadIdx.x == 0) {
        const bool drifted = kickB && !halted;
        unsigned int reb = (drifted && st == 0u && md2 > a.disp_thr2) ? 1u : 0u;
        ctl->rebuild = reb;
        if (drifted) {
            ctl->step = step + 1;
            ctl->last_maxdisp2 = md2;
        }
        if (rec && st == 0u && (mode == IM_LOOP || mode == IM_SAMPLE))
            ctl->obs_count += 1;
        unsigned int loop = 0u;
        if (mode == IM_LOOP) {
            long long rem = remaining - 1, bud = ctl->budget - 1;
            ctl->remaining = rem;
            ctl->budget = bud;
            unsigned int s2 = st;
            if (bud <= 0 && rem > 0) {
                atomicOr(&ctl->status, ST_TIMEOUT);
                s2 |= ST_TIMEOUT;
            }
            loop = (s2 == 0u && rem > 0) ? 1u : 0u;
        }
        ctl->ticket = 0u;
        ctl->n_integrate += 1;
        if (a.use_cond) {
            cudaGraphSetConditional(a.h_rebuild, reb);
            if (mode == IM_LOOP)
                cudaGraphSetConditional(a.h_loop, loop);
        }
    }
}

// ---------------------------------------------------------------------------
// force: pair force, potential and virial over the neighbour list (Sec. 2.2),
// 12-6 potential cut (and shifted) at r_c,ab (Sec. 3, Sec. 5).
// TPP threads share one particle, each taking every TPP-th list entry; the
// lanes' partial sums are combined by shuffles.  MIXED accumulates the force
// with Kahan compensation and combines lanes in double-single (the
// compensated force summation of Sec. 2.4); energies and the virial are
// accumulated only on sample steps and go to per-block FP64 partials.
// ---------------------------------------------------------------------------
template <typename T> struct PairRow {   // parameters of (species i, species j = 0 / 1)
    T rc2[2], sig2[2], eps4[2], eps48[2], shift[2];
};

template <int P, int TPP, bool SAMPLE>
__device__ __forceinline__ void force_impl(const KArgs &a)
{
    __shared__ double sh[32 * 8];
    const int4 b = a.blk_f[blockIdx.x];
    const Rep rp = a.rep[b.z];
    const int lane = threadIdx.x & (TPP - 1);
    const int i = b.x + (int)(threadIdx.x / TPP);
    const bool valid = i < b.y;
    const int ii = valid ? i : b.x;
    const int nn = valid ? a.nnbr[ii] : 0;
    const int *lst = a.nbr + (size_t)ii * (size_t)a.K;

    double acc[8];   // e, virial, wxx, wyy, wzz, wxy, wxz, wyz (lane-0 values, SAMPLE only)
#pragma unroll
    for (int k = 0; k < 8; ++k)
        acc[k] = 0.0;

    if constexpr (P == FP64) {
        const d4 *pos = (const d4 *)a.pa;
        const d4 xi = pos[ii];
        const int ti = species_of(xi.w);
        PairRow<double> pr;
#pragma unroll
        for (int tj = 0; tj < 2; ++tj) {
            pr.rc2[tj] = a.tab.rc2d[ti * 2 + tj];
            pr.sig2[tj] = a.tab.sig2d[ti * 2 + tj];
            pr.eps4[tj] = a.tab.eps4d[ti * 2 + tj];
            pr.eps48[tj] = a.tab.eps48d[ti * 2 + tj];
            pr.shift[tj] = a.tab.shiftd[ti * 2 + tj];
        }
        double fx = 0, fy = 0, fz = 0, en = 0, vir = 0, wxx = 0, wyy = 0, wzz = 0, wxy = 0, wxz = 0, wyz = 0;
        for (int k = lane; k < nn; k += TPP) {
            const int j = __ldg(lst + k);
            const d4 xj = pos[j];
            const int tj = species_of(xj.w);
            const double dx = sep_d(xi.x, xj.x, rp.L, rp.invL);
            const double dy = sep_d(xi.y, xj.y, rp.L, rp.invL);
            const double dz = sep_d(xi.z, xj.z, rp.L, rp.invL);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < pr.rc2[tj]) {
                const double ir2 = 1.0 / r2;
                const double s2 = pr.sig2[tj] * ir2;
                const double s6 = s2 * s2 * s2;
                const double fr = pr.eps48[tj] * ir2 * s6 * (s6 - 0.5);
                fx += fr * dx;
                fy += fr * dy;
                fz += fr * dz;
                if (SAMPLE) {
                    en += pr.eps4[tj] * s6 * (s6 - 1.0) - pr.shift[tj];
                    vir += fr * r2;
                    wxx += fr * dx * dx; wyy += fr * dy * dy; wzz += fr * dz * dz;
                    wxy += fr * dx * dy; wxz += fr * dx * dz; wyz += fr * dy * dz;
                }
            }
        }
#pragma unroll
        for (int o = TPP / 2; o > 0; o >>= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
            if (SAMPLE) {
                en += __shfl_xor_sync(0xffffffffu, en, o);
                vir += __shfl_xor_sync(0xffffffffu, vir, o);
                wxx += __shfl_xor_sync(0xffffffffu, wxx, o);
                wyy += __shfl_xor_sync(0xffffffffu, wyy, o);
                wzz += __shfl_xor_sync(0xffffffffu, wzz, o);
                wxy += __shfl_xor_sync(0xffffffffu, wxy, o);
                wxz += __shfl_xor_sync(0xffffffffu, wxz, o);
                wyz += __shfl_xor_sync(0xffffffffu, wyz, o);
            }
        }
        if (valid && lane == 0) {
            d4 f;
            f.x = fx; f.y = fy; f.z = fz; f.w = SAMPLE ? 0.5 * en : 0.0;
            ((d4 *)a.force)[i] = f;
            if (SAMPLE) {
                acc[0] = 0.5 * en; acc[1] = 0.5 * vir;
                acc[2] = 0.5 * wxx; acc[3] = 0.5 * wyy; acc[4] = 0.5 * wzz;
                acc[5] = 0.5 * wxy; acc[6] = 0.5 * wxz; acc[7] = 0.5 * wyz;
            }
        }
    } else {
        const float4 *pos = (const float4 *)a.pa;
        const float4 Hi = pos[ii];
        float4 li = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (P == MIXED)
            li = ((const float4 *)a.pb)[ii];
        const int ti = species_of(Hi.w);
        PairRow<float> pr;
#pragma unroll
        for (int tj = 0; tj < 2; ++tj) {
            pr.rc2[tj] = a.tab.rc2[ti * 2 + tj];
            pr.sig2[tj] = a.tab.sig2[ti * 2 + tj];
            pr.eps4[tj] = a.tab.eps4[ti * 2 + tj];
            pr.eps48[tj] = a.tab.eps48[ti * 2 + tj];
            pr.shift[tj] = a.tab.shift[ti * 2 + tj];
        }
        float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
        float en = 0.f, vir = 0.f, wxx = 0.f, wyy = 0.f, wzz = 0.f, wxy = 0.f, wxz = 0.f, wyz = 0.f;
        for (int k = lane; k < nn; k += TPP) {
            const int j = __ldg(lst + k);
            const float4 Hj = __ldg(pos + j);
            const int tj = species_of(Hj.w);
            float dx, dy, dz;
            if constexpr (P == MIXED) {
                const float4 lj = __ldg((const float4 *)a.pb + j);
                dx = sep_ds(Hi.x, li.x, Hj.x, lj.x, rp.Lhi, rp.Llo, rp.invLf);
                dy = sep_ds(Hi.y, li.y, Hj.y, lj.y, rp.Lhi, rp.Llo, rp.invLf);
                dz = sep_ds(Hi.z, li.z, Hj.z, lj.z, rp.Lhi, rp.Llo, rp.invLf);
            } else {
                dx = sep_f(Hi.x, Hj.x, rp.Lhi, rp.invLf);
                dy = sep_f(Hi.y, Hj.y, rp.Lhi, rp.invLf);
                dz = sep_f(Hi.z, Hj.z, rp.Lhi, rp.invLf);
            }
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float rc2 = tj ? pr.rc2[1] : pr.rc2[0];
            if (r2 < rc2) {
                const float sig2 = tj ? pr.sig2[1] : pr.sig2[0];
                const float eps48 = tj ? pr.eps48[1] : pr.eps48[0];
                const float ir2 = __frcp_rn(r2);
                const float s2 = sig2 * ir2;
                const float s6 = s2 * s2 * s2;
                const float fr = eps48 * ir2 * s6 * (s6 - 0.5f);
                if constexpr (P == MIXED) {
                    kahan_add(sx, cx, fr * dx);
                    kahan_add(sy, cy, fr * dy);
                    kahan_add(sz, cz, fr * dz);
                } else {
                    sx += fr * dx;
                    sy += fr * dy;
                    sz += fr * dz;
                }
                if (SAMPLE) {
                    const float eps4 = tj ? pr.eps4[1] : pr.eps4[0];
                    const float shift = tj ? pr.shift[1] : pr.shift[0];
                    en += eps4 * s6 * (s6 - 1.0f) - shift;
                    vir += fr * r2;
                    wxx += fr * dx * dx; wyy += fr * dy * dy; wzz += fr * dz * dz;
                    wxy += fr * dx * dy; wxz += fr * dx * dz; wyz += fr * dy * dz;
                }
            }
        }
        // combine the lanes of one particle
        float fx, fy, fz;
        if constexpr (P == MIXED) {
            ds ax = ds_from(sx, -cx), ay = ds_from(sy, -cy), az = ds_from(sz, -cz);
#pragma unroll
            for (int o = TPP / 2; o > 0; o >>= 1) {
                ds bx = ds_from(__shfl_xor_sync(0xffffffffu, ax.hi, o), __shfl_xor_sync(0xffffffffu, ax.lo, o));
                ds by = ds_from(__shfl_xor_sync(0xffffffffu, ay.hi, o), __shfl_xor_sync(0xffffffffu, ay.lo, o));
                ds bz = ds_from(__shfl_xor_sync(0xffffffffu, az.hi, o), __shfl_xor_sync(0xffffffffu, az.lo, o));
                ax = ds_add(ax, bx);
                ay = ds_add(ay, by);
                az = ds_add(az, bz);
            }
            fx = __fadd_rn(ax.hi, ax.lo);
            fy = __fadd_rn(ay.hi, ay.lo);
            fz = __fadd_rn(az.hi, az.lo);
        } else {
#pragma unroll
            for (int o = TPP / 2; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
                sz += __shfl_xor_sync(0xffffffffu, sz, o);
            }
            fx = sx; fy = sy; fz = sz;
        }
        if (SAMPLE) {
            double d[8] = {en, vir, wxx, wyy, wzz, wxy, wxz, wyz};
#pragma unroll
            for (int o = TPP / 2; o > 0; o >>= 1)
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    d[k] += __shfl_xor_sync(0xffffffffu, d[k], o);
            if (valid && lane == 0)
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    acc[k] = 0.5 * d[k];
        }
        if (valid && lane == 0)
            ((float4 *)a.force)[i] = make_float4(fx, fy, fz, SAMPLE ? (float)acc[0] : 0.0f);
    }
    if (SAMPLE) {
        block_sum<8>(acc, sh);
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < 8; ++k)
                a.part_f[(size_t)blockIdx.x * 8 + k] = acc[k];
    }
}

template <int P, int TPP>
__global__ void __launch_bounds__(kForceBlock) k_force(KArgs a)
{
    const Ctl *ctl = a.ctl;
    if (ctl->status)
        return;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd((unsigned long long *)&a.ctl->n_force, 1ull);
    const bool sample = a.fsample || (ctl->step % a.si) == 0;
    if (sample)
        force_impl<P, TPP, true>(a);
    else
        force_impl<P, TPP, false>(a);
}

// ---------------------------------------------------------------------------
// Cell binning by counting sort (Sec. 2.2: integer cell index per particle,
// particles sorted by cell, start index of each cell) with the cells ordered
// along a space-filling curve (the periodic reorder of Sec. 2.2).
// Kernels: k_bin (cell key + histogram) -> k_scan -> k_scatter ->
// k_permute (deterministic order inside a cell, gather of the state) ->
// k_copyback -> k_nbuild.  Each returns at once unless a rebuild is pending.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool rebuild_pending(const Ctl *ctl)
{
    return ctl->status == 0u && ctl->rebuild != 0u;
}

__device__ __forceinline__ int cell_coord(double x, double cscale, int nc)
{
    int c = (int)floor(x * cscale);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__device__ __forceinline__ int cell_coord_f(float x, float cscale, int nc)
{
    int c = (int)floorf(x * cscale);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

template <int P>
__global__ void __launch_bounds__(kIntBlock) k_bin(KArgs a)
{
    Ctl *ctl = a.ctl;
    if (!rebuild_pending(ctl))
        return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->max_nbr = 0;
        atomicAdd((unsigned long long *)&ctl->n_rebuild_k, 1ull);
    }
    const int4 b = a.blk_i[blockIdx.x];
    const int i = b.x + threadIdx.x;
    if (i >= b.y)
        return;
    const Rep rp = a.rep[b.z];
    int cx, cy, cz;
    if constexpr (P == FP64) {
        const d4 x = ((const d4 *)a.pa)[i];
        cx = cell_coord(x.x, rp.cscale, rp.nc);
        cy = cell_coord(x.y, rp.cscale, rp.nc);
        cz = cell_coord(x.z, rp.cscale, rp.nc);
    } else {
        const float4 x = ((const float4 *)a.pa)[i];
        cx = cell_coord_f(x.x, rp.cscalef, rp.nc);
        cy = cell_coord_f(x.y, rp.cscalef, rp.nc);
        cz = cell_coord_f(x.z, rp.cscalef, rp.nc);
    }
    const int key = a.crank[rp.cell0 + (cz * rp.nc + cy) * rp.nc + cx];
    a.key[i] = key;
    atomicAdd(&a.ccount[key], 1);
}

// exclusive scan of the cell histogram by one block; also clears the cursors
template <int P>
__global__ void __launch_bounds__(kScanBlock) k_scan(KArgs a)
{
    __shared__ int wsum[32];
    Ctl *ctl = a.ctl;
    if (!rebuild_pending(ctl))
        return;
    if (threadIdx.x == 0)
        atomicAdd((unsigned long long *)&ctl->n_rebuild_k, 1ull);
    const int n = a.ncell, T = blockDim.x, t = threadIdx.x;
    const int per = (n + T - 1) / T;
    const int s0 = min(t * per, n), s1 = min(s0 + per, n);
    int sum = 0;
    for (int s = s0; s < s1; ++s)
        sum += a.ccount[s];
    const int lane = t & 31, w = t >> 5, nw = T >> 5;
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += y;
    }
    if (lane == 31)
        wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int v = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o)
                v += y;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    int base = (w > 0 ? wsum[w - 1] : 0) + incl - sum;
    for (int s = s0; s < s1; ++s) {
        a.cstart[s] = base;
        base += a.ccount[s];
        a.ccursor[s] = 0;
    }
    if (t == T - 1)
        a.cstart[n] = base;
}

template <int P>
__global__ void __launch_bounds__(kIntBlock) k_scatter(KArgs a)
{
    Ctl *ctl = a.ctl;
    if (!rebuild_pending(ctl))
        return;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd((unsigned long long *)&ctl->n_rebuild_k, 1ull);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n)
        return;
    const int k = a.key[i];
    const int slot = a.cstart[k] + atomicAdd(&a.ccursor[k], 1);
    a.tmpidx[slot] = i;
}

// Final slot of each particle: its cell's start plus the number of particles
// of the same cell with a smaller current index (stable, deterministic), then
// gather of the whole state into the second buffers.
template <int P>
__global__ void __launch_bounds__(kIntBlock) k_permute(KArgs a)
{
    Ctl *ctl = a.ctl;
    if (!rebuild_pending(ctl))
        return;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd((unsigned long long *)&ctl->n_rebuild_k, 1ull);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.n)
        return;
    const int i = a.tmpidx[s];
    const int k = a.key[i];
    const int b0 = a.cstart[k], b1 = a.cstart[k + 1];
    int rank = 0;
    for (int t = b0; t < b1; ++t)
        rank += (a.tmpidx[t] < i) ? 1 : 0;
    const int d = b0 + rank;
    if constexpr (P == FP64) {
        const d4 x = ((const d4 *)a.pa)[i];
        ((d4 *)a.pa2)[d] = x;
        ((d4 *)a.va2)[d] = ((const d4 *)a.va)[i];
        a.rref[d] = make_float4(__double2float_rn(x.x), __double2float_rn(x.y), __double2float_rn(x.z), 0.f);
    } else {
        const float4 x = ((const float4 *)a.pa)[i];
        ((float4 *)a.pa2)[d] = x;
        ((float4 *)a.va2)[d] = ((const float4 *)a.va)[i];
        if constexpr (P == MIXED) {
            ((float4 *)a.pb2)[d] = ((const float4 *)a.pb)[i];
            ((float4 *)a.vb2)[d] = ((const float4 *)a.vb)[i];
        }
        a.rref[d] = make_float4(x.x, x.y, x.z, 0.f);
    }
    a.image2[d] = a.image[i];
    a.cellof[d] = k;
}

template <int P>
__global__ void __launch_bounds__(kIntBlock) k_copyback(KArgs a)
{
    Ctl *ctl = a.ctl;
    if (!rebuild_pending(ctl))
        return;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd((unsigned long long *)&ctl->n_rebuild_k, 1ull);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    for (int c = s; c < a.ncell; c += gridDim.x * blockDim.x)
        a.ccount[c] = 0;
    if (s >= a.n)
        return;
    if constexpr (P == FP64) {
        ((d4 *)a.pa)[s] = ((const d4 *)a.pa2)[s];
        ((d4 *)a.va)[s] = ((const d4 *)a.va2)[s];
    } else {
        ((float4 *)a.pa)[s] = ((const float4 *)a.pa2)[s];
        ((float4 *)a.va)[s] = ((const float4 *)a.va2)[s];
        if constexpr (P == MIXED) {
            ((float4 *)a.pb)[s] = ((const float4 *)a.pb2)[s];
            ((float4 *)a.vb)[s] = ((const float4 *)a.vb2)[s];
        }
    }
    a.image[s] = a.image2[s];
}

// ---------------------------------------------------------------------------
// Neighbour-list build (Sec. 2.2): one warp per particle scans the particles
// of its own and the adjacent cells (27, or all cells when fewer than three
// fit along the box edge) and keeps those closer than r_c,ab + skin (plus a
// rounding margin).  Particle-major list: nbr[i*K + k], coalesced per warp.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kNbBlock) k_nbuild(KArgs a)
{
    Ctl *ctl = a.ctl;
    if (!rebuild_pending(ctl))
        return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd((unsigned long long *)&ctl->n_rebuild_k, 1ull);
        atomicAdd((unsigned long long *)&ctl->rebuilds, 1ull);
    }
    const int lane = threadIdx.x & 31;
    const int i = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (i >= a.n)
        return;   // whole warp
    const int c = a.cellof[i];
    const int4 cc = a.cxyz[c];
    const Rep rp = a.rep[cc.w];
    const int nc = rp.nc;
    const int lo = nc >= 3 ? -1 : 0, hi = nc >= 3 ? 1 : 0;
    int *out = a.nbr + (size_t)i * (size_t)a.K;
    const unsigned lt_mask = (1u << lane) - 1u;
    int cnt = 0;

    // own position
    double xd = 0, yd = 0, zd = 0;
    float4 Hi = make_float4(0.f, 0.f, 0.f, 0.f), li = make_float4(0.f, 0.f, 0.f, 0.f);
    int ti;
    if constexpr (P == FP64) {
        const d4 x = ((const d4 *)a.pa)[i];
        xd = x.x; yd = x.y; zd = x.z;
        ti = species_of(x.w);
    } else {
        Hi = ((const float4 *)a.pa)[i];
        if constexpr (P == MIXED)
            li = ((const float4 *)a.pb)[i];
        ti = species_of(Hi.w);
    }
    for (int dz = lo; dz <= hi; ++dz)
    for (int dy = lo; dy <= hi; ++dy)
    for (int dx = lo; dx <= hi; ++dx) {
        const int x = (cc.x + dx + nc) % nc, y = (cc.y + dy + nc) % nc, z = (cc.z + dz + nc) % nc;
        const int cell = a.crank[rp.cell0 + (z * nc + y) * nc + x];
        const int j0 = a.cstart[cell], j1 = a.cstart[cell + 1];
        for (int jb = j0; jb < j1; jb += 32) {
            const int j = jb + lane;
            bool in = false;
            if (j < j1 && j != i) {
                if constexpr (P == FP64) {
                    const d4 y4 = ((const d4 *)a.pa)[j];
                    const double ex = sep_d(xd, y4.x, rp.L, rp.invL);
                    const double ey = sep_d(yd, y4.y, rp.L, rp.invL);
                    const double ez = sep_d(zd, y4.z, rp.L, rp.invL);
                    in = ex * ex + ey * ey + ez * ez < a.tab.rl2d[ti * 2 + species_of(y4.w)];
                } else {
                    const float4 Hj = ((const float4 *)a.pa)[j];
                    float ex, ey, ez;
                    if constexpr (P == MIXED) {
                        const float4 lj = ((const float4 *)a.pb)[j];
                        ex = sep_ds(Hi.x, li.x, Hj.x, lj.x, rp.Lhi, rp.Llo, rp.invLf);
                        ey = sep_ds(Hi.y, li.y, Hj.y, lj.y, rp.Lhi, rp.Llo, rp.invLf);
                        ez = sep_ds(Hi.z, li.z, Hj.z, lj.z, rp.Lhi, rp.Llo, rp.invLf);
                    } else {
                        ex = sep_f(Hi.x, Hj.x, rp.Lhi, rp.invLf);
                        ey = sep_f(Hi.y, Hj.y, rp.Lhi, rp.invLf);
                        ez = sep_f(Hi.z, Hj.z, rp.Lhi, rp.invLf);
                    }
                    in = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < a.tab.rl2[ti * 2 + species_of(Hj.w)];
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, in);
            const int pre = __popc(m & lt_mask);
            if (in && cnt + pre < a.K)
                out[cnt + pre] = j;
            cnt += __popc(m);
        }
    }
    if (lane == 0) {
        a.nnbr[i] = cnt < a.K ? cnt : a.K;
        atomicMax(&ctl->max_nbr, cnt);
        if (cnt > a.K)
            atomicOr(&ctl->status, ST_OVERFLOW);
    }
}

// ---------------------------------------------------------------------------
// state transfer between the staging area (original order, float64) and the
// working layout; misc. control kernels
// ---------------------------------------------------------------------------
// Load the staged state into slot order = original order, wrap into [0, L),
// split into the precision's representation and request a rebuild.
template <int P>
__global__ void __launch_bounds__(kIntBlock) k_load(KArgs a)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->rebuild = 1u;
        atomicAdd((unsigned long long *)&a.ctl->n_other, 1ull);
    }
    const int4 b = a.blk_i[blockIdx.x];
    const int i = b.x + threadIdx.x;
    if (i >= b.y)
        return;
    const Rep rp = a.rep[b.z];
    const int sp = a.st_code[i];
    double x[3];
    int im[3];
    for (int k = 0; k < 3; ++k) {
        const double v = a.st_pos[3 * (size_t)i + k];
        const double q = floor(v * rp.invL);
        double w = v - q * rp.L;
        int m = a.st_img[3 * (size_t)i + k] + (int)q;
        if (w >= rp.L) { w -= rp.L; m += 1; }
        if (w < 0.0) { w += rp.L; m -= 1; }
        x[k] = w;
        im[k] = m;
    }
    const double *vv = a.st_vel + 3 * (size_t)i;
    if constexpr (P == FP64) {
        d4 p, v;
        p.x = x[0]; p.y = x[1]; p.z = x[2]; p.w = __longlong_as_double((long long)sp);
        v.x = vv[0]; v.y = vv[1]; v.z = vv[2]; v.w = 0.0;
        ((d4 *)a.pa)[i] = p;
        ((d4 *)a.va)[i] = v;
    } else if constexpr (P == MIXED) {
        float H[3], l[3];
        for (int k = 0; k < 3; ++k) {
            // high word on the grid: multiples of rp.grid are exact in float for |x| < 2L
            const double h = rint(x[k] * (double)rp.inv_grid) * (double)rp.grid;
            H[k] = (float)h;
            l[k] = __double2float_rn(x[k] - h);
        }
        ((float4 *)a.pa)[i] = make_float4(H[0], H[1], H[2], __int_as_float(sp));
        ((float4 *)a.pb)[i] = make_float4(l[0], l[1], l[2], 0.f);
        ds vx = ds_from_double(vv[0]), vy = ds_from_double(vv[1]), vz = ds_from_double(vv[2]);
        ((float4 *)a.va)[i] = make_float4(vx.hi, vy.hi, vz.hi, 0.f);
        ((float4 *)a.vb)[i] = make_float4(vx.lo, vy.lo, vz.lo, 0.f);
    } else {
        float fx = __double2float_rn(x[0]), fy = __double2float_rn(x[1]), fz = __double2float_rn(x[2]);
        const float L = rp.Lhi;
        if (fx >= L) fx = 0.f;
        if (fy >= L) fy = 0.f;
        if (fz >= L) fz = 0.f;
        ((float4 *)a.pa)[i] = make_float4(fx, fy, fz, __int_as_float(sp));
        ((float4 *)a.va)[i] = make_float4((float)vv[0], (float)vv[1], (float)vv[2], 0.f);
    }
    a.image[i] = make_int4(im[0], im[1], im[2], i);
}

// Write the state back to the staging area in the original order.
template <int P>
__global__ void __launch_bounds__(kIntBlock) k_getstate(KArgs a)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd((unsigned long long *)&a.ctl->n_other, 1ull);
    if (s >= a.n)
        return;
    const int4 im = a.image[s];
    const size_t t = (size_t)im.w;
    double x[3], v[3];
    if constexpr (P == FP64) {
        const d4 p = ((const d4 *)a.pa)[s], w = ((const d4 *)a.va)[s];
        x[0] = p.x; x[1] = p.y; x[2] = p.z;
        v[0] = w.x; v[1] = w.y; v[2] = w.z;
    } else if constexpr (P == MIXED) {
        const float4 H = ((const float4 *)a.pa)[s], l = ((const float4 *)a.pb)[s];
        const float4 vh = ((const float4 *)a.va)[s], vl = ((const float4 *)a.vb)[s];
        x[0] = (double)H.x + (double)l.x; x[1] = (double)H.y + (double)l.y; x[2] = (double)H.z + (double)l.z;
        v[0] = (double)vh.x + (double)vl.x; v[1] = (double)vh.y + (double)vl.y; v[2] = (double)vh.z + (double)vl.z;
    } else {
        const float4 p = ((const float4 *)a.pa)[s], w = ((const float4 *)a.va)[s];
        x[0] = p.x; x[1] = p.y; x[2] = p.z;
        v[0] = w.x; v[1] = w.y; v[2] = w.z;
    }
    for (int k = 0; k < 3; ++k) {
        a.st_pos[3 * t + k] = x[k];
        a.st_vel[3 * t + k] = v[k];
    }
    a.st_img[3 * t + 0] = im.x;
    a.st_img[3 * t + 1] = im.y;
    a.st_img[3 * t + 2] = im.z;
}

template <int P>
__global__ void __launch_bounds__(kIntBlock) k_expforce(KArgs a)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd((unsigned long long *)&a.ctl->n_other, 1ull);
    if (s >= a.n)
        return;
    const size_t t = (size_t)a.image[s].w;
    double f[4];
    if constexpr (P == FP64) {
        const d4 q = ((const d4 *)a.force)[s];
        f[0] = q.x; f[1] = q.y; f[2] = q.z; f[3] = q.w;
    } else {
        const float4 q = ((const float4 *)a.force)[s];
        f[0] = q.x; f[1] = q.y; f[2] = q.z; f[3] = q.w;
    }
    a.st_f[3 * t + 0] = f[0];
    a.st_f[3 * t + 1] = f[1];
    a.st_f[3 * t + 2] = f[2];
    a.st_e[t] = f[3];
}

// v <- v * scale[replica]  (exact rescale, Sec. 2.3)
template <int P>
__global__ void __launch_bounds__(kIntBlock) k_scale(KArgs a)
{
    if (a.ctl->status)
        return;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd((unsigned long long *)&a.ctl->n_other, 1ull);
    const int4 b = a.blk_i[blockIdx.x];
    const int i = b.x + threadIdx.x;
    if (i >= b.y)
        return;
    const double f = a.scale[b.z];
    if constexpr (P == FP64) {
        d4 v = ((d4 *)a.va)[i];
        v.x *= f; v.y *= f; v.z *= f;
        ((d4 *)a.va)[i] = v;
    } else if constexpr (P == MIXED) {
        const ds fs = ds_from_double(f);
        float4 vh = ((float4 *)a.va)[i], vl = ((float4 *)a.vb)[i];
        ds x = ds_mul(ds_from(vh.x, vl.x), fs), y = ds_mul(ds_from(vh.y, vl.y), fs),
           z = ds_mul(ds_from(vh.z, vl.z), fs);
        ((float4 *)a.va)[i] = make_float4(x.hi, y.hi, z.hi, 0.f);
        ((float4 *)a.vb)[i] = make_float4(x.lo, y.lo, z.lo, 0.f);
    } else {
        float4 v = ((float4 *)a.va)[i];
        const float ff = (float)f;
        v.x *= ff; v.y *= ff; v.z *= ff;
        ((float4 *)a.va)[i] = v;
    }
}

template <int P>
__global__ void k_set_steps(KArgs a)
{
    a.ctl->remaining = a.nsteps;
    a.ctl->budget = a.nsteps + 2;
    a.ctl->n_other += 1;
}

// clear a reported status so that the handle can be inspected and reused
template <int P>
__global__ void k_reset(KArgs a)
{
    a.ctl->status = 0u;
    a.ctl->ticket = 0u;
    a.ctl->maxdisp2 = 0u;
    a.ctl->remaining = 0;
    a.ctl->n_other += 1;
}

// request a list rebuild before the next force evaluation
template <int P>
__global__ void k_mark_rebuild(KArgs a)
{
    a.ctl->rebuild = 1u;
    a.ctl->n_other += 1;
}

template <int P>
KernelSet make_kernel_set()
{
    KernelSet k;
    k.integrate = (const void *)k_integrate<P>;
    k.force[0] = (const void *)k_force<P, 1>;
    k.force[1] = (const void *)k_force<P, 2>;
    k.force[2] = (const void *)k_force<P, 4>;
    k.force[3] = (const void *)k_force<P, 8>;
    k.force[4] = (const void *)k_force<P, 16>;
    k.force[5] = (const void *)k_force<P, 32>;
    k.bin = (const void *)k_bin<P>;
    k.scan = (const void *)k_scan<P>;
    k.scatter = (const void *)k_scatter<P>;
    k.permute = (const void *)k_permute<P>;
    k.copyback = (const void *)k_copyback<P>;
    k.nbuild = (const void *)k_nbuild<P>;
    k.load = (const void *)k_load<P>;
    k.getstate = (const void *)k_getstate<P>;
    k.expforce = (const void *)k_expforce<P>;
    k.scale = (const void *)k_scale<P>;
    k.set_steps = (const void *)k_set_steps<P>;
    k.reset = (const void *)k_reset<P>;
    k.mark_rebuild = (const void *)k_mark_rebuild<P>;
    return k;
}

}  // namespace mdk
