// md_kernels.cuh -- the MD step kernels, templated on the precision mode.
//
// Included by one translation unit per precision (md_kernels_{fp64,mixed,fp32}.cu),
// each of which instantiates every kernel for its mode and exports a table of
// kernel entry addresses.  All kernels take one KArgs by value.
//
// State layout in device memory (slot order = cell order after each rebuild):
//   MIXED  pos: float4 (H.x, H.y, H.z, species bits) + float4 (l.x, l.y, l.z, 0);
//               position = H + l with H on a power-of-two grid (see anchor_wrap)
//          vel: float4 high words + float4 low words (normalised double-single)
//   FP64   pos: d4 (x, y, z, species bits), vel: d4
//   FP32   pos: float4 (x, y, z, species bits), vel: float4
//   force: float4 (MIXED, FP32) or d4 (FP64): (Fx, Fy, Fz, e_i)
//   image: int4 (nx, ny, nz, original index)
// Positions are double-buffered (Ctl::pos_par): the step kernel reads the
// current buffer for every neighbour and writes the drifted positions into the
// other one.  Velocities and images are double-buffered by Ctl::state_par,
// which changes only when a rebuild permutes the particles.
//
// One MD step = one launch of k_step: pair forces over the neighbour list,
// then, per particle, the velocity-Verlet half kick that completes v(t), the
// kinetic sample, the half kick that starts the next step and the drift
// (Sec. 2.2).  Its last block finishes the reductions and decides, with a
// bound on how far particles can move before the next check, whether the
// lists must be rebuilt (the displacement criterion of Sec. 2.2).
#pragma once

#include <type_traits>

#include "md_common.cuh"

namespace mdk {

constexpr int kIntBlock = 256;   // per-particle kernels: one thread per particle
constexpr int kForceBlock = 128; // force / step kernels: tpp threads per particle
constexpr int kNbCells = 4;      // neighbour build, warp per cell: cells per block
constexpr int kNbBlock = 32 * kNbCells;
constexpr int kNbBlockB = 256;   // neighbour build, block per cell: threads per block
constexpr int kScanBlock = 1024;
constexpr int kScanPer = 8;      // cell counts per thread and tile of the scan
constexpr int kPartF = 12;       // doubles per block partial of the force / step kernels
constexpr int kUnr = 8;          // list entries per lane and iteration of the FP32 pair loops
                                 // (a multiple of 4, at most 8: lists are padded to 8)
constexpr int kPfDepth = 1;      // iterations ahead at which the list indices are loaded
constexpr bool kSplitUpdate = false; // below 4 lanes: one lane updates (measured faster than sharing)

// Bounds-checked build (compile with -DMD_CHECK_BOUNDS=1; off in the product
// library): every index read from device memory (list entries, cell keys,
// permutation slots) is tested against its array before use.
#ifndef MD_CHECK_BOUNDS
#define MD_CHECK_BOUNDS 0
#endif
constexpr bool kCheckBounds = MD_CHECK_BOUNDS != 0;

// i unchanged if 0 <= i < n; otherwise (checked builds) ST_BOUNDS is recorded
// and `safe` returned, so that the access stays inside the array.
__device__ __forceinline__ int checked(const KArgs &a, int i, int n, int safe)
{
    if constexpr (kCheckBounds) {
        if ((unsigned int)i >= (unsigned int)n) {
            atomicOr(&a.ctl->status, ST_BOUNDS);
            return safe;
        }
    }
    return i;
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

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

// Maxima of three non-negative floats over the block; valid in thread 0.
__device__ __forceinline__ void block_max3(float &a, float &b, float &c, float *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    a = warp_max(a);
    b = warp_max(b);
    c = warp_max(c);
    if (lane == 0) {
        sh[3 * w] = a;
        sh[3 * w + 1] = b;
        sh[3 * w + 2] = c;
    }
    __syncthreads();
    if (w == 0) {
        a = warp_max(lane < nw ? sh[3 * lane] : 0.f);
        b = warp_max(lane < nw ? sh[3 * lane + 1] : 0.f);
        c = warp_max(lane < nw ? sh[3 * lane + 2] : 0.f);
    }
    __syncthreads();
}

// Maxima of three non-negative floats and the sum of one double over the
// block, valid in thread 0, with one pair of barriers.  The sum takes the
// same steps as component 0 of block_sum (so a per-step potential energy
// equals the one of a sample record bit for bit).
__device__ __forceinline__ void block_max3_sum1(float &a, float &b, float &c, double &e, float *shf, double *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    a = warp_max(a);
    b = warp_max(b);
    c = warp_max(c);
    e = warp_sum(e);
    if (lane == 0) {
        shf[3 * w] = a;
        shf[3 * w + 1] = b;
        shf[3 * w + 2] = c;
        sh[w] = e;
    }
    __syncthreads();
    if (w == 0) {
        a = warp_max(lane < nw ? shf[3 * lane] : 0.f);
        b = warp_max(lane < nw ? shf[3 * lane + 1] : 0.f);
        c = warp_max(lane < nw ? shf[3 * lane + 2] : 0.f);
        e = warp_sum(lane < nw ? sh[lane] : 0.0);
    }
    __syncthreads();
}

// The same with the energy sum in double-single (FP32 arithmetic): warps add
// by shuffles in a fixed butterfly order, then warp 0 adds the warps' sums.
// shf: 3 * 32 + 2 * 32 floats.
__device__ __forceinline__ void block_max3_sum1(float &a, float &b, float &c, ds &e, float *shf, double *)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    a = warp_max(a);
    b = warp_max(b);
    c = warp_max(c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        e = ds_add(e, ds_from(__shfl_xor_sync(0xffffffffu, e.hi, o), __shfl_xor_sync(0xffffffffu, e.lo, o)));
    if (lane == 0) {
        shf[3 * w] = a;
        shf[3 * w + 1] = b;
        shf[3 * w + 2] = c;
        shf[96 + 2 * w] = e.hi;
        shf[97 + 2 * w] = e.lo;
    }
    __syncthreads();
    if (w == 0) {
        a = warp_max(lane < nw ? shf[3 * lane] : 0.f);
        b = warp_max(lane < nw ? shf[3 * lane + 1] : 0.f);
        c = warp_max(lane < nw ? shf[3 * lane + 2] : 0.f);
        e = lane < nw ? ds_from(shf[96 + 2 * lane], shf[97 + 2 * lane]) : ds_from(0.f, 0.f);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            e = ds_add(e, ds_from(__shfl_xor_sync(0xffffffffu, e.hi, o), __shfl_xor_sync(0xffffffffu, e.lo, o)));
    }
    __syncthreads();
}

__device__ __forceinline__ int species_of(float w) { return __float_as_int(w) & 15; }
__device__ __forceinline__ int species_of(double w) { return (int)(__double_as_longlong(w) & 15); }

// buffer selection by parity
__device__ __forceinline__ void *pos_a(const KArgs &a, int par) { return par ? a.pa2 : a.pa; }
__device__ __forceinline__ void *pos_b(const KArgs &a, int par) { return par ? a.pb2 : a.pb; }
__device__ __forceinline__ void *vel_a(const KArgs &a, int par) { return par ? a.va2 : a.va; }
__device__ __forceinline__ void *vel_b(const KArgs &a, int par) { return par ? a.vb2 : a.vb; }
__device__ __forceinline__ int4 *img_of(const KArgs &a, int par) { return par ? a.image2 : a.image; }

// Re-anchor a double-single coordinate so that its high word lies on the grid
// of spacing `grid` (a power of two chosen so that every coordinate in
// [-L, 2L) is exactly representable on it), then wrap it into [0, L).
// Shifting an anchored high word by the anchored box edge Lhi is exact in
// single precision, so the wrap loses nothing; differences of high words are
// exact too (the displacement check uses them).  The pair loops read the
// fixed-point copy instead (fixq).  Returns the change of the image counter
// (-1, 0, 1).
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

// Fixed-point position (MIXED): x / L in units of 2^-32, modulo 2^32, from
// the exact double value of a double-single coordinate.  The periodic box is
// the full 32-bit circle, so the 32-bit wrapped difference of two coordinates
// is the minimum-image separation, exact in integers; only its conversion to
// single precision rounds.  One unit is L / 2^32 (8.8e-9 sigma at L = 38).
//
// Without FP64 (whose pipe is narrow on this GPU): the high word is an
// integer number m of grid steps (0 <= m < 2^24, exact), so x 2^32 / L =
// m C + l 2^32 / L with C = grid 2^32 / L in (2^9, 2^10].  m C is formed in
// 64-bit integers from C in units of 2^-28 (error < 2^-5 units) and rounded;
// |l| <= grid, so l 2^32 / L (at most C, single precision, error < 2^-13
// units) is rounded on its own.  The result is within 1 + 2^-5 units of the
// exact value (two roundings), the same in every kernel.
__device__ __forceinline__ unsigned int fixq(float H, float l, const Rep &rp)
{
    const unsigned int m = (unsigned int)__float2int_rn(__fmul_rn(H, rp.inv_grid));   // exact
    const unsigned long long hi = ((unsigned long long)m * rp.qgrid + (1ull << 27)) >> 28;
    return (unsigned int)hi + (unsigned int)__float2int_rn(__fmul_rn(l, rp.qscale));
}

__device__ __forceinline__ float sep_q(unsigned int qi, unsigned int qj, float unit)
{
    return __int2float_rn((int)(qi - qj)) * unit;
}

__device__ __forceinline__ int4 *q_of(const KArgs &a, int par) { return par ? a.qb : a.qa; }

// Kahan-compensated accumulation: the running sum is s - c.
__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    float y = __fsub_rn(x, c);
    float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// Smoothing of Sec. 4: U = V g(x), g(x) = x^4 / (1 + x^4), x = (r - r_c) / (h sigma_ab).
// On entry fr = -V'(r)/r and v = V(r); on exit fr = -U'(r)/r and v = U(r):
//   -U'/r = (-V'/r) g - V g'(x) / (h sigma r),  g'(x) = 4 x^3 / (1 + x^4)^2.
__device__ __forceinline__ void smooth_pair(float r2, float rc, float ihs, float &fr, float &v)
{
    const float rinv = rsqrtf(r2);
    const float x = (r2 * rinv - rc) * ihs;
    const float x2 = x * x, x4 = x2 * x2;
    const float den = __fdividef(1.0f, 1.0f + x4);
    const float g = x4 * den;
    const float dg = 4.0f * x2 * x * den * den;
    fr = fr * g - v * dg * ihs * rinv;
    v = v * g;
}

__device__ __forceinline__ void smooth_pair(double r2, double rc, double ihs, double &fr, double &v)
{
    const double r = sqrt(r2);
    const double x = (r - rc) * ihs;
    const double x2 = x * x, x4 = x2 * x2;
    const double den = 1.0 / (1.0 + x4);
    const double g = x4 * den;
    const double dg = 4.0 * x2 * x * den * den;
    fr = fr * g - v * dg * ihs / r;
    v = v * g;
}

template <int P> using FT = typename std::conditional<P == FP64, double, float>::type;

// Per-particle potential energy and its block sums: double in FP64 mode,
// double-single (FP32 arithmetic) otherwise, so that the every-step energy
// reduction adds no FP64 instruction to the single-precision modes.
template <int P> using ET = typename std::conditional<P == FP64, double, ds>::type;
__device__ __forceinline__ double e_value(double e) { return e; }
__device__ __forceinline__ double e_value(ds e) { return ds_to_double(e); }
__device__ __forceinline__ float e_float(double e) { return (float)e; }
__device__ __forceinline__ float e_float(ds e) { return __fadd_rn(e.hi, e.lo); }
template <int P> __device__ __forceinline__ ET<P> e_zero()
{
    if constexpr (P == FP64)
        return 0.0;
    else
        return ds_from(0.f, 0.f);
}

// ---------------------------------------------------------------------------
// Per-particle velocity-Verlet pieces (Sec. 2.2), in the precision's state
// representation: MIXED updates velocities and positions in double-single
// (Sec. 2.4), FP64 in double, FP32 in float.
// ---------------------------------------------------------------------------
template <int P> struct PState;
template <> struct PState<MIXED> { float4 H, l; ds vx, vy, vz; int sp; };
template <> struct PState<FP64> { d4 x; double vx, vy, vz; int sp; };
template <> struct PState<FP32> { float4 x; float vx, vy, vz; int sp; };

template <int P>
__device__ __forceinline__ void load_pos(const KArgs &a, int pp, int i, PState<P> &s)
{
    if constexpr (P == MIXED) {
        s.H = ((const float4 *)pos_a(a, pp))[i];
        s.l = ((const float4 *)pos_b(a, pp))[i];
        s.sp = species_of(s.H.w);
    } else if constexpr (P == FP64) {
        s.x = ((const d4 *)pos_a(a, pp))[i];
        s.sp = species_of(s.x.w);
    } else {
        s.x = ((const float4 *)pos_a(a, pp))[i];
        s.sp = species_of(s.x.w);
    }
}

template <int P>
__device__ __forceinline__ void load_vel(const KArgs &a, int sp, int i, PState<P> &s)
{
    if constexpr (P == MIXED) {
        const float4 h = ((const float4 *)vel_a(a, sp))[i], l = ((const float4 *)vel_b(a, sp))[i];
        s.vx = ds_from(h.x, l.x);
        s.vy = ds_from(h.y, l.y);
        s.vz = ds_from(h.z, l.z);
    } else if constexpr (P == FP64) {
        const d4 v = ((const d4 *)vel_a(a, sp))[i];
        s.vx = v.x; s.vy = v.y; s.vz = v.z;
    } else {
        const float4 v = ((const float4 *)vel_a(a, sp))[i];
        s.vx = v.x; s.vy = v.y; s.vz = v.z;
    }
}

template <int P>
__device__ __forceinline__ void store_vel(const KArgs &a, int sp, int i, const PState<P> &s)
{
    if constexpr (P == MIXED) {
        ((float4 *)vel_a(a, sp))[i] = make_float4(s.vx.hi, s.vy.hi, s.vz.hi, 0.f);
        ((float4 *)vel_b(a, sp))[i] = make_float4(s.vx.lo, s.vy.lo, s.vz.lo, 0.f);
    } else if constexpr (P == FP64) {
        d4 v;
        v.x = s.vx; v.y = s.vy; v.z = s.vz; v.w = 0.0;
        ((d4 *)vel_a(a, sp))[i] = v;
    } else {
        ((float4 *)vel_a(a, sp))[i] = make_float4(s.vx, s.vy, s.vz, 0.f);
    }
}

// v += dt/(2m) f
template <int P>
__device__ __forceinline__ void half_kick(const KArgs &a, PState<P> &s, FT<P> fx, FT<P> fy, FT<P> fz)
{
    if constexpr (P == MIXED) {
        const ds hk = ds_from(a.hdtm_hi[s.sp], a.hdtm_lo[s.sp]);
        s.vx = ds_add(s.vx, ds_mul_f(hk, fx));
        s.vy = ds_add(s.vy, ds_mul_f(hk, fy));
        s.vz = ds_add(s.vz, ds_mul_f(hk, fz));
    } else if constexpr (P == FP64) {       // (roundings spelled out: the same in every kernel)
        const double hk = a.hdtm[s.sp];
        s.vx = fma(hk, fx, s.vx);
        s.vy = fma(hk, fy, s.vy);
        s.vz = fma(hk, fz, s.vz);
    } else {
        const float hk = a.hdtm_hi[s.sp];
        s.vx = fmaf(hk, fx, s.vx);
        s.vy = fmaf(hk, fy, s.vy);
        s.vz = fmaf(hk, fz, s.vz);
    }
}

// kinetic energy and momentum of the particle in FP64: kin[0..3]
template <int P>
__device__ __forceinline__ void kinetic(const KArgs &a, const PState<P> &s, double *kin)
{
    double vx, vy, vz;
    if constexpr (P == MIXED) {
        vx = ds_to_double(s.vx); vy = ds_to_double(s.vy); vz = ds_to_double(s.vz);
    } else {
        vx = s.vx; vy = s.vy; vz = s.vz;
    }
    const double m = a.mass[s.sp];
    kin[0] = __dmul_rn(0.5 * m, fma(vz, vz, fma(vy, vy, __dmul_rn(vx, vx))));
    kin[1] = m * vx;
    kin[2] = m * vy;
    kin[3] = m * vz;
}

// |v|^2 and |d|^2 feed the rebuild decision, which sets the particle order and
// so the summation order: their roundings are spelled out, so that every
// kernel that computes them decides alike.
__device__ __forceinline__ float norm2f(float x, float y, float z)
{
    return fmaf(z, z, fmaf(y, y, __fmul_rn(x, x)));
}
__device__ __forceinline__ float norm2(float x, float y, float z) { return norm2f(x, y, z); }
__device__ __forceinline__ float norm2(double x, double y, double z)
{
    return (float)fma(z, z, fma(y, y, __dmul_rn(x, x)));
}
__device__ __forceinline__ float speed2(const PState<MIXED> &s) { return norm2f(s.vx.hi, s.vy.hi, s.vz.hi); }
__device__ __forceinline__ float speed2(const PState<FP64> &s) { return norm2(s.vx, s.vy, s.vz); }
__device__ __forceinline__ float speed2(const PState<FP32> &s) { return norm2f(s.vx, s.vy, s.vz); }

// r += dt v, wrapped into [0, L) with image counting; writes the new position
// into buffer `dst`, updates the image counter in the state buffers `spar`,
// returns the squared displacement since the last list build.
template <int P>
__device__ __forceinline__ float drift(const KArgs &a, const Rep &rp, PState<P> &s, int dst, int spar, int i,
                                       unsigned int &bad)
{
    int ix, iy, iz;
    float dd;
    if constexpr (P == MIXED) {
        const ds dt = ds_from(a.dt_hi, a.dt_lo);
        const ds sx = ds_mul(dt, s.vx), sy = ds_mul(dt, s.vy), sz = ds_mul(dt, s.vz);
        const float lim = 0.25f * rp.Lhi;
        if (fabsf(sx.hi) > lim || fabsf(sy.hi) > lim || fabsf(sz.hi) > lim)
            bad |= ST_UNSTABLE;
        const ds nx = ds_add(ds_from(s.H.x, s.l.x), sx);
        const ds ny = ds_add(ds_from(s.H.y, s.l.y), sy);
        const ds nz = ds_add(ds_from(s.H.z, s.l.z), sz);
        ix = anchor_wrap(nx, rp.grid, rp.inv_grid, rp.Lhi, rp.Llo, s.H.x, s.l.x);
        iy = anchor_wrap(ny, rp.grid, rp.inv_grid, rp.Lhi, rp.Llo, s.H.y, s.l.y);
        iz = anchor_wrap(nz, rp.grid, rp.inv_grid, rp.Lhi, rp.Llo, s.H.z, s.l.z);
        if (!isfinite(s.H.x) || !isfinite(s.H.y) || !isfinite(s.H.z))
            bad |= ST_NONFINITE;
        ((float4 *)pos_a(a, dst))[i] = s.H;
        ((float4 *)pos_b(a, dst))[i] = s.l;
        q_of(a, dst)[i] = make_int4((int)fixq(s.H.x, s.l.x, rp), (int)fixq(s.H.y, s.l.y, rp),
                                    (int)fixq(s.H.z, s.l.z, rp), s.sp);
        const float4 rr = a.rref[i];
        const float ex = __fadd_rn(sep_f(s.H.x, rr.x, rp.Lhi, rp.invLf), s.l.x);
        const float ey = __fadd_rn(sep_f(s.H.y, rr.y, rp.Lhi, rp.invLf), s.l.y);
        const float ez = __fadd_rn(sep_f(s.H.z, rr.z, rp.Lhi, rp.invLf), s.l.z);
        dd = norm2f(ex, ey, ez);
    } else if constexpr (P == FP64) {
        const double sx = __dmul_rn(a.dt, s.vx), sy = __dmul_rn(a.dt, s.vy), sz = __dmul_rn(a.dt, s.vz);
        const double lim = 0.25 * rp.L;
        if (fabs(sx) > lim || fabs(sy) > lim || fabs(sz) > lim)
            bad |= ST_UNSTABLE;
        double x = __dadd_rn(s.x.x, sx), y = __dadd_rn(s.x.y, sy), z = __dadd_rn(s.x.z, sz);
        ix = iy = iz = 0;
        if (x >= rp.L) { x -= rp.L; ix = 1; } else if (x < 0.0) { x += rp.L; ix = -1; }
        if (y >= rp.L) { y -= rp.L; iy = 1; } else if (y < 0.0) { y += rp.L; iy = -1; }
        if (z >= rp.L) { z -= rp.L; iz = 1; } else if (z < 0.0) { z += rp.L; iz = -1; }
        if (!isfinite(x) || !isfinite(y) || !isfinite(z))
            bad |= ST_NONFINITE;
        s.x.x = x; s.x.y = y; s.x.z = z;
        ((d4 *)pos_a(a, dst))[i] = s.x;
        const float4 rr = a.rref[i];
        const float ex = sep_f(__double2float_rn(x), rr.x, rp.Lhi, rp.invLf);
        const float ey = sep_f(__double2float_rn(y), rr.y, rp.Lhi, rp.invLf);
        const float ez = sep_f(__double2float_rn(z), rr.z, rp.Lhi, rp.invLf);
        dd = norm2f(ex, ey, ez);
    } else {
        const float dt = a.dt_hi;
        const float sx = __fmul_rn(dt, s.vx), sy = __fmul_rn(dt, s.vy), sz = __fmul_rn(dt, s.vz);
        const float L = rp.Lhi;
        if (fabsf(sx) > 0.25f * L || fabsf(sy) > 0.25f * L || fabsf(sz) > 0.25f * L)
            bad |= ST_UNSTABLE;
        float x = __fadd_rn(s.x.x, sx), y = __fadd_rn(s.x.y, sy), z = __fadd_rn(s.x.z, sz);
        ix = iy = iz = 0;
        if (x >= L) { x -= L; ix = 1; } else if (x < 0.f) { x += L; ix = -1; }
        if (y >= L) { y -= L; iy = 1; } else if (y < 0.f) { y += L; iy = -1; }
        if (z >= L) { z -= L; iz = 1; } else if (z < 0.f) { z += L; iz = -1; }
        // a coordinate just below 0 can round to L when wrapped: it is 0 of the
        // original image
        if (x >= L) { x = 0.f; ix += 1; }
        if (y >= L) { y = 0.f; iy += 1; }
        if (z >= L) { z = 0.f; iz += 1; }
        if (!isfinite(x) || !isfinite(y) || !isfinite(z))
            bad |= ST_NONFINITE;
        s.x.x = x; s.x.y = y; s.x.z = z;
        ((float4 *)pos_a(a, dst))[i] = s.x;
        const float4 rr = a.rref[i];
        const float ex = sep_f(x, rr.x, L, rp.invLf);
        const float ey = sep_f(y, rr.y, L, rp.invLf);
        const float ez = sep_f(z, rr.z, L, rp.invLf);
        dd = norm2f(ex, ey, ez);
    }
    if (ix | iy | iz) {
        int4 *im = img_of(a, spar);
        int4 q = im[i];
        q.x += ix;
        q.y += iy;
        q.z += iz;
        im[i] = q;
    }
    return dd;
}

// ---------------------------------------------------------------------------
// reductions finished by the last block of a step / integrate kernel
// ---------------------------------------------------------------------------
__device__ __forceinline__ void write_record(const KArgs &a, int mode, int r, const double *v, long long step,
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
    if (mode == IM_LOOP || mode == IM_SAMPLE)
        a.epot[(step % a.epot_cap) * a.nrep + r] = v[0];
    if (mode == IM_TOTALS)
        a.totals[r] = o;
    else if (mode == IM_KE) {
        const Rep &rp = a.rep[r];
        double dof = 3.0 * (double)rp.n - 3.0;
        double target = a.scale[r];
        a.scale[r] = (v[8] > 0.0) ? sqrt(target * dof / (2.0 * v[8])) : 1.0;
    } else
        a.ring[slot * a.nrep + r] = o;
}

// Potential-energy partial sums, one per warp of the force / step kernels
// (part_e): double in FP64 mode, double-single elsewhere, so that the every-
// step energy reduction costs no FP64 arithmetic in the single-precision
// modes.  Two sets, by the parity of the step the energies belong to, so that
// a step's partials survive the next step until they are added up.
constexpr int kWarpsF = kForceBlock / 32;

template <int P>
__device__ __forceinline__ size_t epart_index(const KArgs &a, long long step, int chunk, int warp)
{
    return (size_t)(step & 1) * (size_t)a.nblk_f * kWarpsF + (size_t)chunk * kWarpsF + warp;
}

template <int P>
__device__ __forceinline__ void put_epart(const KArgs &a, size_t k, ET<P> e)
{
    if constexpr (P == FP64)
        ((double *)a.part_e)[k] = e;
    else
        ((float2 *)a.part_e)[k] = make_float2(e.hi, e.lo);
}

template <int P>
__device__ __forceinline__ ET<P> get_epart(const KArgs &a, size_t k)
{
    if constexpr (P == FP64) {
        return ((const double *)a.part_e)[k];
    } else {
        const float2 x = ((const float2 *)a.part_e)[k];
        return ds_from(x.x, x.y);
    }
}

__device__ __forceinline__ double e_add(double x, double y) { return x + y; }
__device__ __forceinline__ ds e_add(ds x, ds y) { return ds_add(x, y); }

__device__ __forceinline__ double e_warp_sum(double e) { return warp_sum(e); }
__device__ __forceinline__ ds e_warp_sum(ds e)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        e = ds_add(e, ds_from(__shfl_xor_sync(0xffffffffu, e.hi, o), __shfl_xor_sync(0xffffffffu, e.lo, o)));
    return e;
}

// The warp's energy sum into its partial of step `step`.  Every lane of the
// warp calls it (the sum is a full-warp shuffle); lane 0 writes if `write`.
template <int P>
__device__ __forceinline__ void store_warp_energy(const KArgs &a, long long step, int chunk, ET<P> e, bool write)
{
    e = e_warp_sum(e);
    if ((threadIdx.x & 31) == 0 && write)
        put_epart<P>(a, epart_index<P>(a, step, chunk, threadIdx.x >> 5), e);
}

// Potential energy of one replica at `step` from its warps' partials, by the
// whole block: thread t adds partials p0 + t, p0 + t + blockDim, ... in that
// order (eight loads in flight), then the threads' sums are added in a fixed
// tree.  Valid in thread 0.  Every thread of the block must call it.
template <int P>
__device__ double epot_sum_block(const KArgs &a, const Rep &rp, long long step, float *shf, double *sh)
{
    ET<P> v = e_zero<P>();
    const int stride = blockDim.x;
    const size_t base = epart_index<P>(a, step, 0, 0);
    int b = rp.bf0 * kWarpsF + threadIdx.x;
    const int end = rp.bf1 * kWarpsF;
    for (; b + 7 * stride < end; b += 8 * stride) {
        ET<P> x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            x[u] = get_epart<P>(a, base + b + u * stride);
#pragma unroll
        for (int u = 0; u < 8; ++u)
            v = e_add(v, x[u]);
    }
    for (; b < end; b += stride)
        v = e_add(v, get_epart<P>(a, base + b));
    float d0 = 0.f, d1 = 0.f, d2 = 0.f;
    block_max3_sum1(d0, d1, d2, v, shf, sh);
    return e_value(v);
}

// The same by one thread, for handles with many replicas (one thread each).
template <int P>
__device__ double epot_sum_seq(const KArgs &a, const Rep &rp, long long step)
{
    ET<P> v = e_zero<P>();
    const size_t base = epart_index<P>(a, step, 0, 0);
    for (int b = rp.bf0 * kWarpsF; b < rp.bf1 * kWarpsF; ++b)
        v = e_add(v, get_epart<P>(a, base + b));
    return e_value(v);
}

// Per-replica sums of the block partials, in a fixed order (deterministic).
// Potential-side values come from part_f[.][1..7] and the energy sums
// part_e; kinetic values from part_f[.][8..11] (step kernel, from_f = true)
// or part_i[.][0..3].
template <int P>
__device__ void finish_reductions(const KArgs &a, int mode, bool from_f, long long step, float md2, double *sh,
                                  float *shf)
{
    const Ctl *ctl = a.ctl;
    const long long slot = ctl->obs_count % (long long)a.obs_cap;
    const long long rebuilds = ctl->rebuilds;
    const bool want_f = mode != IM_KE;
    if (a.nrep <= 8) {
        for (int r = 0; r < a.nrep; ++r) {
            const Rep rp = a.rep[r];
            double v[12];
#pragma unroll
            for (int k = 0; k < 12; ++k)
                v[k] = 0.0;
            if (want_f || from_f)
                for (int b = rp.bf0 + threadIdx.x; b < rp.bf1; b += blockDim.x)
#pragma unroll
                    for (int k = 1; k < kPartF; ++k)
                        v[k] += a.part_f[(size_t)b * kPartF + k];
            if (!from_f) {
#pragma unroll
                for (int k = 8; k < 12; ++k)
                    v[k] = 0.0;
                for (int b = rp.bi0 + threadIdx.x; b < rp.bi1; b += blockDim.x)
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        v[8 + k] += a.part_i[(size_t)b * 4 + k];
            }
            block_sum<12>(v, sh);
            const double e = want_f ? epot_sum_block<P>(a, rp, step, shf, sh) : 0.0;
            if (threadIdx.x == 0) {
                v[0] = e;
                write_record(a, mode, r, v, step, md2, rebuilds, slot);
            }
        }
    } else {
        for (int r = threadIdx.x; r < a.nrep; r += blockDim.x) {
            const Rep rp = a.rep[r];
            double v[12];
            for (int k = 0; k < 12; ++k)
                v[k] = 0.0;
            if (want_f || from_f)
                for (int b = rp.bf0; b < rp.bf1; ++b)
                    for (int k = 1; k < kPartF; ++k)
                        v[k] += a.part_f[(size_t)b * kPartF + k];
            if (!from_f) {
                for (int k = 8; k < 12; ++k)
                    v[k] = 0.0;
                for (int b = rp.bi0; b < rp.bi1; ++b)
                    for (int k = 0; k < 4; ++k)
                        v[8 + k] += a.part_i[(size_t)b * 4 + k];
            }
            if (want_f)
                v[0] = epot_sum_seq<P>(a, rp, step);
            write_record(a, mode, r, v, step, md2, rebuilds, slot);
        }
        __syncthreads();
    }
}

// The potential energy of every replica at `step` (a step that recorded no
// sample) into the per-step series: the same sums as finish_reductions takes.
// Run by one whole block.
template <int P>
__device__ void finish_epot(const KArgs &a, long long step, double *sh, float *shf)
{
    const long long slot = step % a.epot_cap;
    if (a.nrep <= 8) {
        for (int r = 0; r < a.nrep; ++r) {
            const double e = epot_sum_block<P>(a, a.rep[r], step, shf, sh);
            if (threadIdx.x == 0)
                a.epot[slot * a.nrep + r] = e;
        }
    } else {
        for (int r = threadIdx.x; r < a.nrep; r += blockDim.x)
            a.epot[slot * a.nrep + r] = epot_sum_seq<P>(a, a.rep[r], step);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        a.epot_step[slot] = step;
}

// Rebuild decision: the list built at the last rebuild holds every pair
// within r_c + skin, so it stays complete while no particle has moved more
// than skin/2.  The next check comes after `look` further drifts, each at
// most dt (v + look dt a) per particle: rebuild now if the largest
// displacement plus that bound could exceed skin/2 (with a rounding margin).
__device__ __forceinline__ unsigned int need_rebuild(const KArgs &a, float md2, float mv2, float ma2)
{
    const float ahead = (float)a.lookahead * (float)a.dt * (sqrtf(mv2) + 2.0f * (float)a.lookahead *
                                                                              (float)a.dt * sqrtf(ma2));
    const float d = sqrtf(md2) + ahead;
    return d > a.disp_thr ? 1u : 0u;
}

// ---------------------------------------------------------------------------
// pair forces over the neighbour list (Sec. 2.2), 12-6 potential cut (and
// shifted) at r_c,ab (Sec. 3, Sec. 5).  TPP threads share one particle; each
// lane takes groups of consecutive list entries (16-byte index loads) and
// issues their gathers together.  List rows are padded with the particle
// itself to whole groups of 8 (r^2 = 0 exactly: never inside), so the loops
// carry no end-of-row masks.  Single precision: a group's contributions are
// summed branch-free (zero factor outside the cutoff) and the group sum enters
// a Kahan accumulator (MIXED; plain sum for FP32); lanes are combined in
// double-single.  The pair potential is summed alongside, every step (the
// potential energy is a per-step reduction of Sec. 2.2).  On return every lane
// of the particle holds the total force and ep, half the sum of its pair
// energies; the virial comes from pair_energy on sample steps.
// ---------------------------------------------------------------------------
// 1/24 as a double-single pair (the accumulated energies are 12 V; a particle
// takes half of each pair)
constexpr float kE24hi = (float)(1.0 / 24.0);
constexpr float kE24lo = (float)(1.0 / 24.0 - (double)(float)(1.0 / 24.0));

template <typename T> struct PairRow {   // parameters of (species i, species j = 0 / 1)
    T rc2[2], sig2[2], eps4[2], eps48[2], shift[2], rc[2], ihs[2], c[2];
};

template <int P, int TPP, bool SM>
__device__ __forceinline__ void pair_forces(const KArgs &a, const Rep &rp, int pp, int ii, int nn,
                                            FT<P> &fx, FT<P> &fy, FT<P> &fz, ET<P> &ep)
{
    const int lane = threadIdx.x & (TPP - 1);
    const int *lst = a.nbr + (size_t)ii * (size_t)a.Kstride;
    if constexpr (P == FP64) {
        const d4 *pos = (const d4 *)pos_a(a, pp);
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
            pr.rc[tj] = a.tab.rcd[ti * 2 + tj];
            pr.ihs[tj] = a.tab.ihsd[ti * 2 + tj];
            pr.c[tj] = a.tab.vcd[ti * 2 + tj];
        }
        double sx = 0, sy = 0, sz = 0, se = 0;          // se: sum of 12 V
        for (int k0 = 4 * lane; k0 < nn; k0 += 4 * TPP) {
            const int4 q = __ldg((const int4 *)(lst + k0));
            const int jj[4] = {q.x, q.y, q.z, q.w};
            d4 xs[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)                 // padded rows: whole groups
                xs[u] = pos[checked(a, jj[u], a.n, ii)];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const d4 xj = xs[u];
                const int tj = species_of(xj.w);
                const double dx = sep_d(xi.x, xj.x, rp.L, rp.invL);
                const double dy = sep_d(xi.y, xj.y, rp.L, rp.invL);
                const double dz = sep_d(xi.z, xj.z, rp.L, rp.invL);
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 < pr.rc2[tj] && r2 > 0.0) {          // r2 = 0: the padding entry
                    const double ir2 = 1.0 / r2;
                    const double s2 = pr.sig2[tj] * ir2;
                    const double s6 = s2 * s2 * s2;
                    double fr = pr.eps48[tj] * ir2 * s6 * (s6 - 0.5);
                    if (SM) {
                        double v = pr.eps4[tj] * s6 * (s6 - 1.0) - pr.shift[tj];
                        smooth_pair(r2, pr.rc[tj], pr.ihs[tj], fr, v);
                        se = fma(12.0, v, se);
                    } else {
                        se = fma(pr.eps48[tj], fma(s6, s6, -(s6 + pr.c[tj])), se);
                    }
                    sx += fr * dx;
                    sy += fr * dy;
                    sz += fr * dz;
                }
            }
        }
#pragma unroll
        for (int o = TPP / 2; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
            sz += __shfl_xor_sync(0xffffffffu, sz, o);
            se += __shfl_xor_sync(0xffffffffu, se, o);
        }
        fx = sx; fy = sy; fz = sz;
        ep = se * (1.0 / 24.0);
    } else {
        // MIXED reads the fixed-point copy (16 B per neighbour), FP32 the positions
        const float4 *pos = (const float4 *)pos_a(a, pp);
        const int4 *qp = q_of(a, pp);
        float4 Hi = make_float4(0.f, 0.f, 0.f, 0.f);
        int4 Qi = make_int4(0, 0, 0, 0);
        int ti;
        if constexpr (P == MIXED) {
            Qi = qp[ii];
            ti = Qi.w;
        } else {
            Hi = pos[ii];
            ti = species_of(Hi.w);
        }
        PairRow<float> pr;
#pragma unroll
        for (int tj = 0; tj < 2; ++tj) {
            pr.rc2[tj] = a.tab.rc2[ti * 2 + tj];
            pr.sig2[tj] = a.tab.sig2[ti * 2 + tj];
            pr.eps4[tj] = a.tab.eps4[ti * 2 + tj];
            pr.eps48[tj] = a.tab.eps48[ti * 2 + tj];
            pr.shift[tj] = a.tab.shift[ti * 2 + tj];
            pr.rc[tj] = a.tab.rc[ti * 2 + tj];
            pr.ihs[tj] = a.tab.ihs[ti * 2 + tj];
            pr.c[tj] = a.tab.vc[ti * 2 + tj];
        }
        // the energy is accumulated as 12 V = eps48_ab (s6^2 - s6 - c_ab), c_ab = S_ab / (4 eps_ab):
        // eps48, masked by the cutoff test, serves the force and the energy alike
        float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f, se = 0.f, ce = 0.f;
        // list indices are loaded kPfDepth iterations ahead, so that only the
        // position gathers remain on each iteration's critical path
        // (K is a multiple of 8: every 16-byte index load is in bounds and aligned)
        constexpr int kStride = kUnr * TPP;
        int4 pf[kPfDepth][kUnr / 4];
#pragma unroll
        for (int d = 0; d < kPfDepth; ++d)
#pragma unroll
            for (int w = 0; w < kUnr / 4; ++w) {
                const int k = kUnr * lane + d * kStride;
                pf[d][w] = k < nn ? __ldg((const int4 *)(lst + k + 4 * w)) : make_int4(0, 0, 0, 0);
            }
        for (int k0 = kUnr * lane; k0 < nn; k0 += kStride) {
            int jj[kUnr];
#pragma unroll
            for (int w = 0; w < kUnr / 4; ++w) {
                const int4 q = pf[0][w];
                jj[4 * w] = q.x;
                jj[4 * w + 1] = q.y;
                jj[4 * w + 2] = q.z;
                jj[4 * w + 3] = q.w;
            }
#pragma unroll
            for (int d = 0; d + 1 < kPfDepth; ++d)
#pragma unroll
                for (int w = 0; w < kUnr / 4; ++w)
                    pf[d][w] = pf[d + 1][w];
            if (k0 + kPfDepth * kStride < nn)
#pragma unroll
                for (int w = 0; w < kUnr / 4; ++w)
                    pf[kPfDepth - 1][w] = __ldg((const int4 *)(lst + k0 + kPfDepth * kStride + 4 * w));
            float4 Hs[kUnr];
            int4 Qs[kUnr];
#pragma unroll
            for (int u = 0; u < kUnr; ++u) {
                // rows are padded with the particle itself up to a multiple of kUnr
                const int j = checked(a, jj[u], a.n, ii);
                if constexpr (P == MIXED)
                    Qs[u] = __ldg(qp + j);
                else
                    Hs[u] = __ldg(pos + j);
            }
            float gx = 0.f, gy = 0.f, gz = 0.f, gv = 0.f;
#pragma unroll
            for (int u = 0; u < kUnr; ++u) {
                int tj;
                float dx, dy, dz;
                if constexpr (P == MIXED) {
                    const int4 Qj = Qs[u];
                    tj = Qj.w;
                    dx = sep_q(Qi.x, Qj.x, rp.qunit);
                    dy = sep_q(Qi.y, Qj.y, rp.qunit);
                    dz = sep_q(Qi.z, Qj.z, rp.qunit);
                } else {
                    const float4 Hj = Hs[u];
                    tj = species_of(Hj.w);
                    dx = sep_f(Hi.x, Hj.x, rp.Lhi, rp.invLf);
                    dy = sep_f(Hi.y, Hj.y, rp.Lhi, rp.invLf);
                    dz = sep_f(Hi.z, Hj.z, rp.Lhi, rp.invLf);
                }
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                // (the particle itself, r2 = 0 exactly, is never inside)
                const bool in = r2 > 0.0f && r2 < (tj ? pr.rc2[1] : pr.rc2[0]);
                const float sig2 = tj ? pr.sig2[1] : pr.sig2[0];
                const float e48 = in ? (tj ? pr.eps48[1] : pr.eps48[0]) : 0.0f;
                const float ir2 = __fdividef(1.0f, in ? r2 : 1.0f);
                const float s2 = sig2 * ir2;
                const float s6 = s2 * s2 * s2;
                float fr = e48 * ir2 * s6 * (s6 - 0.5f);
                if (SM) {
                    const float eps4 = tj ? pr.eps4[1] : pr.eps4[0];
                    const float shift = tj ? pr.shift[1] : pr.shift[0];
                    float v = in ? fmaf(eps4, s6 * s6 - s6, -shift) : 0.0f;
                    smooth_pair(in ? r2 : 1.0f, tj ? pr.rc[1] : pr.rc[0], tj ? pr.ihs[1] : pr.ihs[0], fr, v);
                    gv = fmaf(12.0f, v, gv);
                } else {
                    const float c = tj ? pr.c[1] : pr.c[0];
                    gv = fmaf(e48, fmaf(s6, s6, -(s6 + c)), gv);
                }
                gx = fmaf(fr, dx, gx);
                gy = fmaf(fr, dy, gy);
                gz = fmaf(fr, dz, gz);
            }
            if constexpr (P == MIXED) {
                kahan_add(sx, cx, gx);
                kahan_add(sy, cy, gy);
                kahan_add(sz, cz, gz);
                kahan_add(se, ce, gv);
            } else {
                sx += gx;
                sy += gy;
                sz += gz;
                se += gv;
            }
        }
        if constexpr (P == MIXED) {
            ds ax = ds_from(sx, -cx), ay = ds_from(sy, -cy), az = ds_from(sz, -cz), ae = ds_from(se, -ce);
#pragma unroll
            for (int o = TPP / 2; o > 0; o >>= 1) {
                ds bx = ds_from(__shfl_xor_sync(0xffffffffu, ax.hi, o), __shfl_xor_sync(0xffffffffu, ax.lo, o));
                ds by = ds_from(__shfl_xor_sync(0xffffffffu, ay.hi, o), __shfl_xor_sync(0xffffffffu, ay.lo, o));
                ds bz = ds_from(__shfl_xor_sync(0xffffffffu, az.hi, o), __shfl_xor_sync(0xffffffffu, az.lo, o));
                ds be = ds_from(__shfl_xor_sync(0xffffffffu, ae.hi, o), __shfl_xor_sync(0xffffffffu, ae.lo, o));
                ax = ds_add(ax, bx);
                ay = ds_add(ay, by);
                az = ds_add(az, bz);
                ae = ds_add(ae, be);
            }
            fx = __fadd_rn(ax.hi, ax.lo);
            fy = __fadd_rn(ay.hi, ay.lo);
            fz = __fadd_rn(az.hi, az.lo);
            ep = ds_mul(ae, ds_from(kE24hi, kE24lo));         // half of the sum of V = (12 V) / 24
        } else {
#pragma unroll
            for (int o = TPP / 2; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
                sz += __shfl_xor_sync(0xffffffffu, sz, o);
                se += __shfl_xor_sync(0xffffffffu, se, o);
            }
            fx = sx; fy = sy; fz = sz;
            ep = ds_from(se * (1.0f / 24.0f), 0.f);
        }
    }
}

// Virial and virial tensor of particle ii (half of each pair, the less
// frequent reductions of Sec. 2.2), as a separate pass over the list on sample
// steps so that the every-step loop carries no virial accumulators.
// acc[1..7] = W, W_xx, W_yy, W_zz, W_xy, W_xz, W_yz; acc[0] is left as it is.
template <int P, int TPP, bool SM>
__device__ __forceinline__ void pair_virial(const KArgs &a, const Rep &rp, int pp, int ii, int nn, double *acc)
{
    const int lane = threadIdx.x & (TPP - 1);
    const int *lst = a.nbr + (size_t)ii * (size_t)a.Kstride;
    FT<P> d7[7] = {0, 0, 0, 0, 0, 0, 0};
    if constexpr (P == FP64) {
        const d4 *pos = (const d4 *)pos_a(a, pp);
        const d4 xi = pos[ii];
        const int ti = species_of(xi.w);
        for (int k = lane; k < nn; k += TPP) {
            const d4 xj = pos[checked(a, __ldg(lst + k), a.n, ii)];
            const int ab = ti * 2 + species_of(xj.w);
            const double dx = sep_d(xi.x, xj.x, rp.L, rp.invL);
            const double dy = sep_d(xi.y, xj.y, rp.L, rp.invL);
            const double dz = sep_d(xi.z, xj.z, rp.L, rp.invL);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < a.tab.rc2d[ab] && r2 > 0.0) {
                const double ir2 = 1.0 / r2;
                const double s2 = a.tab.sig2d[ab] * ir2;
                const double s6 = s2 * s2 * s2;
                double fr = a.tab.eps48d[ab] * ir2 * s6 * (s6 - 0.5);
                if (SM) {
                    double v = a.tab.eps4d[ab] * s6 * (s6 - 1.0) - a.tab.shiftd[ab];
                    smooth_pair(r2, a.tab.rcd[ab], a.tab.ihsd[ab], fr, v);
                }
                d7[0] += fr * r2;
                d7[1] += fr * dx * dx; d7[2] += fr * dy * dy; d7[3] += fr * dz * dz;
                d7[4] += fr * dx * dy; d7[5] += fr * dx * dz; d7[6] += fr * dy * dz;
            }
        }
    } else {
        const int4 *qp = q_of(a, pp);
        const float4 *pos = (const float4 *)pos_a(a, pp);
        int4 Qi = make_int4(0, 0, 0, 0);
        float4 Hi = make_float4(0.f, 0.f, 0.f, 0.f);
        int ti;
        if constexpr (P == MIXED) {
            Qi = qp[ii];
            ti = Qi.w;
        } else {
            Hi = pos[ii];
            ti = species_of(Hi.w);
        }
        for (int k = lane; k < nn; k += TPP) {
            const int j = checked(a, __ldg(lst + k), a.n, ii);
            float dx, dy, dz;
            int ab;
            if constexpr (P == MIXED) {
                const int4 Qj = __ldg(qp + j);
                ab = ti * 2 + Qj.w;
                dx = sep_q(Qi.x, Qj.x, rp.qunit);
                dy = sep_q(Qi.y, Qj.y, rp.qunit);
                dz = sep_q(Qi.z, Qj.z, rp.qunit);
            } else {
                const float4 Hj = __ldg(pos + j);
                ab = ti * 2 + species_of(Hj.w);
                dx = sep_f(Hi.x, Hj.x, rp.Lhi, rp.invLf);
                dy = sep_f(Hi.y, Hj.y, rp.Lhi, rp.invLf);
                dz = sep_f(Hi.z, Hj.z, rp.Lhi, rp.invLf);
            }
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (r2 < a.tab.rc2[ab] && r2 > 0.0f) {
                const float ir2 = __fdividef(1.0f, r2);
                const float s2 = a.tab.sig2[ab] * ir2;
                const float s6 = s2 * s2 * s2;
                float fr = a.tab.eps48[ab] * ir2 * s6 * (s6 - 0.5f);
                if (SM) {
                    float v = a.tab.eps4[ab] * s6 * (s6 - 1.0f) - a.tab.shift[ab];
                    smooth_pair(r2, a.tab.rc[ab], a.tab.ihs[ab], fr, v);
                }
                d7[0] += fr * r2;
                d7[1] += fr * dx * dx; d7[2] += fr * dy * dy; d7[3] += fr * dz * dz;
                d7[4] += fr * dx * dy; d7[5] += fr * dx * dz; d7[6] += fr * dy * dz;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        double v = (double)d7[k];
#pragma unroll
        for (int o = TPP / 2; o > 0; o >>= 1)
            v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[1 + k] = 0.5 * v;
    }
}

template <int P, typename E>
__device__ __forceinline__ void store_force(const KArgs &a, int i, FT<P> fx, FT<P> fy, FT<P> fz, E e)
{
    if constexpr (P == FP64) {
        d4 f;
        f.x = fx; f.y = fy; f.z = fz; f.w = e_value(e);
        ((d4 *)a.force)[i] = f;
    } else {
        ((float4 *)a.force)[i] = make_float4(fx, fy, fz, e_float(e));
    }
}

// ---------------------------------------------------------------------------
// k_force: forces (and on request the potential-side reductions) at the
// current positions; used when a handle is created or its state replaced and
// by md_compute_forces.
// ---------------------------------------------------------------------------
template <int P, int TPP, bool SAMPLE, bool SM>
__device__ __forceinline__ void force_only(const KArgs &a)
{
    __shared__ double sh[32 * kPartF];
    const Ctl *ctl = a.ctl;
    const int pp = ctl->pos_par;
    const int4 b = a.blk_f[blockIdx.x];
    const Rep rp = a.rep[b.z];
    const int lane = threadIdx.x & (TPP - 1);
    const int i = b.x + (int)(threadIdx.x / TPP);
    const bool valid = i < b.y;
    const int ii = valid ? i : b.x;
    const int nn = valid ? a.nnbr[ii] : 0;
    FT<P> fx, fy, fz;
    ET<P> ep;
    double acc[kPartF];
#pragma unroll
    for (int k = 0; k < kPartF; ++k)
        acc[k] = 0.0;
    pair_forces<P, TPP, SM>(a, rp, pp, ii, nn, fx, fy, fz, ep);
    acc[0] = e_value(ep);
    if (SAMPLE)
        pair_virial<P, TPP, SM>(a, rp, pp, ii, nn, acc);
    if (!(valid && lane == 0)) {
#pragma unroll
        for (int k = 0; k < kPartF; ++k)
            acc[k] = 0.0;
    }
    if (valid && lane == 0)
        store_force<P>(a, i, fx, fy, fz, ep);
    if (SAMPLE) {
        store_warp_energy<P>(a, ctl->step, b.w, (valid && lane == 0) ? ep : e_zero<P>(), true);
        block_sum<kPartF>(acc, sh);
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < kPartF; ++k)
                a.part_f[(size_t)b.w * kPartF + k] = acc[k];
    }
}

template <int P, int TPP, bool SM>
__global__ void __launch_bounds__(kForceBlock) k_force(KArgs a)
{
    const Ctl *ctl = a.ctl;
    if (ctl->status)
        return;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd((unsigned long long *)&a.ctl->n_force, 1ull);
    if (a.fsample || (ctl->step % a.si) == 0)
        force_only<P, TPP, true, SM>(a);
    else
        force_only<P, TPP, false, SM>(a);
}

// ---------------------------------------------------------------------------
// k_step: one whole MD step.  Positions r(t) (current buffer), forces f(t)
// from the list, then per particle: v(t) = v(t-1/2) + dt/2m f(t) [sample],
// and unless this is the last step of md_step: v(t+1/2) = v(t) + dt/2m f(t),
// r(t+1) = r(t) + dt v(t+1/2) into the other buffer.  Last block: step
// counter, buffer flip, sample record, rebuild decision, graph conditions.
// ---------------------------------------------------------------------------
// One Cartesian component of the velocity-Verlet update, done by lane c of
// the particle's group: half kick(s), drift, re-anchor / wrap, displacement
// from the build position.  vh/vl: velocity component (hi/lo for MIXED, vh
// alone otherwise); returns the squared displacement component.
template <int P>
__device__ __forceinline__ void component_update(const KArgs &a, const Rep &rp, int pp, int spar, int i, int c,
                                                 int sp, float f_c, double f_cd, bool sample, bool last,
                                                 float &vh, float &vl, double &vd, float rr,
                                                 double &ke, double &pc, float &dd, float &vv, unsigned int &bad)
{
    const size_t e = 4 * (size_t)i + c;
    if constexpr (P == MIXED) {
        const ds hk = ds_from(a.hdtm_hi[sp], a.hdtm_lo[sp]);
        ds v = ds_add(ds_from(vh, vl), ds_mul_f(hk, f_c));
        if (sample) {
            const double x = ds_to_double(v);
            ke = 0.5 * a.mass[sp] * x * x;
            pc = a.mass[sp] * x;
        }
        if (!last) {
            v = ds_add(v, ds_mul_f(hk, f_c));
            const ds s = ds_mul(ds_from(a.dt_hi, a.dt_lo), v);
            if (fabsf(s.hi) > 0.25f * rp.Lhi)
                bad |= ST_UNSTABLE;
            const float H = ((const float *)pos_a(a, pp))[e], l = ((const float *)pos_b(a, pp))[e];
            float Hn, ln;
            const int dimg = anchor_wrap(ds_add(ds_from(H, l), s), rp.grid, rp.inv_grid, rp.Lhi, rp.Llo, Hn, ln);
            if (!isfinite(Hn))
                bad |= ST_NONFINITE;
            ((float *)pos_a(a, pp ^ 1))[e] = Hn;
            ((float *)pos_b(a, pp ^ 1))[e] = ln;
            ((unsigned int *)q_of(a, pp ^ 1))[e] = fixq(Hn, ln, rp);
            const float dx = __fadd_rn(sep_f(Hn, rr, rp.Lhi, rp.invLf), ln);
            dd = dx * dx;
            vv = v.hi * v.hi;
            if (dimg)
                ((int *)img_of(a, spar))[e] += dimg;
        }
        vh = v.hi;
        vl = v.lo;
    } else if constexpr (P == FP64) {
        const double hk = a.hdtm[sp];            // (roundings spelled out, as in half_kick / drift)
        double v = fma(hk, f_cd, vd);
        if (sample) {
            ke = 0.5 * a.mass[sp] * v * v;
            pc = a.mass[sp] * v;
        }
        if (!last) {
            v = fma(hk, f_cd, v);
            const double s = __dmul_rn(a.dt, v);
            if (fabs(s) > 0.25 * rp.L)
                bad |= ST_UNSTABLE;
            double x = __dadd_rn(((const double *)pos_a(a, pp))[e], s);
            int dimg = 0;
            if (x >= rp.L) { x -= rp.L; dimg = 1; } else if (x < 0.0) { x += rp.L; dimg = -1; }
            if (!isfinite(x))
                bad |= ST_NONFINITE;
            ((double *)pos_a(a, pp ^ 1))[e] = x;
            const float dx = sep_f(__double2float_rn(x), rr, rp.Lhi, rp.invLf);
            dd = dx * dx;
            vv = (float)(v * v);
            if (dimg)
                ((int *)img_of(a, spar))[e] += dimg;
        }
        vd = v;
    } else {
        const float hk = a.hdtm_hi[sp];
        float v = fmaf(hk, f_c, vh);
        if (sample) {
            ke = 0.5 * a.mass[sp] * (double)v * (double)v;
            pc = a.mass[sp] * (double)v;
        }
        if (!last) {
            v = fmaf(hk, f_c, v);
            const float s = __fmul_rn(a.dt_hi, v);
            const float L = rp.Lhi;
            if (fabsf(s) > 0.25f * L)
                bad |= ST_UNSTABLE;
            float x = __fadd_rn(((const float *)pos_a(a, pp))[e], s);
            int dimg = 0;
            if (x >= L) { x -= L; dimg = 1; } else if (x < 0.f) { x += L; dimg = -1; }
            if (x >= L) { x = 0.f; dimg += 1; }
            if (!isfinite(x))
                bad |= ST_NONFINITE;
            ((float *)pos_a(a, pp ^ 1))[e] = x;
            const float dx = sep_f(x, rr, L, rp.invLf);
            dd = dx * dx;
            vv = v * v;
            if (dimg)
                ((int *)img_of(a, spar))[e] += dimg;
        }
        vh = v;
    }
}

// Step body: after the pair loop the lanes of a particle's group share its
// update.  Lane l owns the components c = l*NC .. l*NC + NC - 1 (NC = 1 for 4
// or more lanes, 4 / TPP below): c = 0..2 are the Cartesian components of the
// double-single kick-drift-kick, c = 3 carries the species word to the new
// position buffer.  The operands of the update are loaded before the
// neighbour loop so that their latency is hidden.
template <int P, int TPP, bool SAMPLE, bool SM>
__device__ __forceinline__ void step_body_split(const KArgs &a, const int4 *tab, int row, bool active, bool last,
                                                int pp, int spar, double *part, ET<P> &eo, float &d2, float &v2, float &a2,
                                                unsigned int &bad)
{
    constexpr int NC = TPP >= 4 ? 1 : 4 / TPP;
    const int4 b = tab[row];
    const Rep rp = a.rep[b.z];
    const int lane = threadIdx.x & (TPP - 1);
    const int i = b.x + (int)(threadIdx.x / TPP);
    const bool valid = active && i < b.y;
    const int ii = (i < b.y) ? i : b.x;
    const int nn = valid ? a.nnbr[ii] : 0;
    float vh[NC], vl[NC], rr[NC];
    double vd[NC];
#pragma unroll
    for (int u = 0; u < NC; ++u) {
        const int c = lane * NC + u;
        const size_t e = 4 * (size_t)ii + (c < 3 ? c : 0);
        vh[u] = 0.f; vl[u] = 0.f; rr[u] = 0.f; vd[u] = 0.0;
        if (valid && c < 3) {
            if constexpr (P == FP64) {
                vd[u] = ((const double *)vel_a(a, spar))[e];
            } else {
                vh[u] = ((const float *)vel_a(a, spar))[e];
                if constexpr (P == MIXED)
                    vl[u] = ((const float *)vel_b(a, spar))[e];
            }
            rr[u] = ((const float *)a.rref)[e];
        }
    }
    FT<P> fx = 0, fy = 0, fz = 0;
    ET<P> ep = e_zero<P>();
#pragma unroll
    for (int k = 0; k < kPartF; ++k)
        part[k] = 0.0;
    eo = e_zero<P>();
    pair_forces<P, TPP, SM>(a, rp, pp, ii, nn, fx, fy, fz, ep);
    if (SAMPLE)
        pair_virial<P, TPP, SM>(a, rp, pp, ii, nn, part);
    // Every lane of the warp must reach the shuffles below, including the
    // lanes of padding particles past the end of a replica's range: they skip
    // the update and contribute zeros.
    int sp = 0;
    if (valid) {
        if constexpr (P == FP64)
            sp = species_of(((const double *)pos_a(a, pp))[4 * (size_t)i + 3]);
        else
            sp = species_of(((const float *)pos_a(a, pp))[4 * (size_t)i + 3]);
    }
    if (valid && lane == 0)
        store_force<P>(a, i, fx, fy, fz, ep);
    double ke = 0.0, p3[3] = {0.0, 0.0, 0.0};
    float dd = 0.f, vv = 0.f;
#pragma unroll
    for (int u = 0; u < NC; ++u) {
        const int c = lane * NC + u;
        if (!valid) {
            // no update
        } else if (c < 3) {
            const size_t e = 4 * (size_t)i + c;
            const FT<P> f_c = c == 0 ? fx : (c == 1 ? fy : fz);
            double kc = 0.0, pc = 0.0;
            float dc = 0.f, wc = 0.f;
            component_update<P>(a, rp, pp, spar, i, c, sp, (float)f_c, (double)f_c, SAMPLE, last, vh[u], vl[u],
                                vd[u], rr[u], kc, pc, dc, wc, bad);
            ke += kc;
            dd += dc;
            vv += wc;
            p3[0] += c == 0 ? pc : 0.0;
            p3[1] += c == 1 ? pc : 0.0;
            p3[2] += c == 2 ? pc : 0.0;
            if constexpr (P == FP64) {
                ((double *)vel_a(a, spar))[e] = vd[u];
            } else {
                ((float *)vel_a(a, spar))[e] = vh[u];
                if constexpr (P == MIXED)
                    ((float *)vel_b(a, spar))[e] = vl[u];
            }
        } else if (c == 3 && !last) {
            // the species word travels with the position
            if constexpr (P == FP64)
                ((double *)pos_a(a, pp ^ 1))[4 * (size_t)i + 3] = ((const double *)pos_a(a, pp))[4 * (size_t)i + 3];
            else
                ((float *)pos_a(a, pp ^ 1))[4 * (size_t)i + 3] = ((const float *)pos_a(a, pp))[4 * (size_t)i + 3];
            if constexpr (P == MIXED)
                ((int *)q_of(a, pp ^ 1))[4 * (size_t)i + 3] = sp;
        }
    }
    // combine the component lanes (the first min(TPP, 4) lanes of the group)
#pragma unroll
    for (int o = (TPP < 4 ? TPP : 4) / 2; o > 0; o >>= 1) {
        dd += __shfl_xor_sync(0xffffffffu, dd, o);
        vv += __shfl_xor_sync(0xffffffffu, vv, o);
        if (SAMPLE) {
            ke += __shfl_xor_sync(0xffffffffu, ke, o);
            p3[0] += __shfl_xor_sync(0xffffffffu, p3[0], o);
            p3[1] += __shfl_xor_sync(0xffffffffu, p3[1], o);
            p3[2] += __shfl_xor_sync(0xffffffffu, p3[2], o);
        }
    }
    if (!valid || lane != 0) {
#pragma unroll
        for (int k = 0; k < kPartF; ++k)
            part[k] = 0.0;
        return;
    }
    eo = ep;
    if (SAMPLE) {
        part[8] = ke;
        part[9] = p3[0];
        part[10] = p3[1];
        part[11] = p3[2];
    }
    if (!last) {
        d2 = dd;
        v2 = vv;
        const float im = a.inv_mass[sp];
        a2 = __fmul_rn(__fmul_rn(norm2(fx, fy, fz), im), im);
    }
}

template <int P, int TPP, bool SAMPLE, bool SM>
__device__ __forceinline__ void step_body(const KArgs &a, const int4 *tab, int row, bool active, bool last,
                                          int pp, int spar, double *part, ET<P> &eo, float &d2, float &v2, float &a2,
                                          unsigned int &bad)
{
    if constexpr (kSplitUpdate || TPP >= 4) {
        step_body_split<P, TPP, SAMPLE, SM>(a, tab, row, active, last, pp, spar, part, eo, d2, v2, a2, bad);
        return;
    }
    const int4 b = tab[row];
    const Rep rp = a.rep[b.z];
    const int lane = threadIdx.x & (TPP - 1);
    const int i = b.x + (int)(threadIdx.x / TPP);
    const bool valid = active && i < b.y;
    const int ii = (i < b.y) ? i : b.x;
    const int nn = valid ? a.nnbr[ii] : 0;
    FT<P> fx = 0, fy = 0, fz = 0;
    ET<P> ep = e_zero<P>();
#pragma unroll
    for (int k = 0; k < kPartF; ++k)
        part[k] = 0.0;
    eo = e_zero<P>();
    pair_forces<P, TPP, SM>(a, rp, pp, ii, nn, fx, fy, fz, ep);
    if (SAMPLE)
        pair_virial<P, TPP, SM>(a, rp, pp, ii, nn, part);
    if (!(valid && lane == 0)) {
#pragma unroll
        for (int k = 0; k < kPartF; ++k)
            part[k] = 0.0;
        return;
    }
    eo = ep;
    store_force<P>(a, i, fx, fy, fz, ep);
    PState<P> s;
    load_pos<P>(a, pp, i, s);
    load_vel<P>(a, spar, i, s);
    half_kick<P>(a, s, fx, fy, fz);                 // completes v(t)
    if (SAMPLE)
        kinetic<P>(a, s, part + 8);
    if (!last) {
        half_kick<P>(a, s, fx, fy, fz);             // v(t + 1/2)
        d2 = drift<P>(a, rp, s, pp ^ 1, spar, i, bad);
        v2 = speed2(s);
        const float im = a.inv_mass[s.sp];
        a2 = __fmul_rn(__fmul_rn(norm2(fx, fy, fz), im), im);
    }
    store_vel<P>(a, spar, i, s);
}

// Blocks per SM the unsmoothed single-precision step kernels are compiled for:
// 7 x 128 threads at <= 72 registers, so that a 1024-block launch (KA N=65536
// at 2 lanes per particle) is a single wave on 152 SMs.  FP64 and the smoothed
// kernels keep the compiler's own register choice (they would spill).
template <int P, bool SM> constexpr int step_min_blocks() { return (P != FP64 && !SM) ? 7 : 0; }

template <int P, int TPP, bool SM, bool SWEEP>
__global__ void __launch_bounds__(kForceBlock, step_min_blocks<P, SM>()) k_step(KArgs a)
{
    __shared__ double sh[32 * kPartF];
    __shared__ float shf[160];
    __shared__ int s_last, s_first;
    __shared__ float s_m[4];
    Ctl *ctl = a.ctl;
    const unsigned int st0 = ctl->status;
    const long long step = ctl->step;
    const long long remaining = ctl->remaining;
    const long long pend = ctl->epot_pending;   // an earlier step whose energies await their sum
    const int pp = ctl->pos_par, spar = ctl->state_par;
    // The status word can change while the launch runs (another block's atomicOr),
    // so threads of one block may read different values: it gates only per-particle
    // work.  Everything that shapes the block's barriers and the lanes' shuffles
    // (sample) depends on fields that change only in the last block.
    const bool active = st0 == 0u && remaining > 0;
    const bool last = remaining == 1;
    const bool sample = remaining > 0 && (step % a.si) == 0;
    if (threadIdx.x == 0)                       // device timing of this launch: earliest start
        atomicMax(&ctl->t_first_inv, ~global_ns());

    if constexpr (SWEEP) {
        // The block sweeps its run of chunks: rows blockIdx.x * cpb ... of the
        // step table.  Per chunk: this step's potential energy, one partial per
        // warp (written only by active launches, so that an idle one never
        // overwrites partials that still await their sum; the shuffles run in
        // every lane regardless); block maxima into the launch's maxima every
        // step; the chunk's other reductions on sample steps (component 0 stays
        // unused).
        for (int q = 0; q < a.cpb; ++q) {
            const int row = blockIdx.x * a.cpb + q;
            const int chunk = a.blk_s[row].w;
            if (chunk < 0)                       // (padding rows: the same for the whole block)
                break;
            double part[kPartF];
            ET<P> eo;
            float d2 = 0.f, v2 = 0.f, a2 = 0.f;
            unsigned int bad = 0u;
            if (sample)
                step_body<P, TPP, true, SM>(a, a.blk_s, row, active, last, pp, spar, part, eo, d2, v2, a2,
                                            bad);
            else
                step_body<P, TPP, false, SM>(a, a.blk_s, row, active, last, pp, spar, part, eo, d2, v2, a2,
                                             bad);
            if (bad)
                atomicOr(&ctl->status, bad);
            store_warp_energy<P>(a, step, chunk, eo, active);
            block_max3(d2, v2, a2, shf);
            if (sample)
                block_sum<kPartF>(part, sh);
            if (threadIdx.x == 0) {
                if (sample) {
                    const size_t pb = (size_t)chunk * kPartF;
#pragma unroll
                    for (int k = 1; k < kPartF; ++k)
                        a.part_f[pb + k] = part[k];
                }
                if (d2 > 0.f)
                    atomicMax(&ctl->maxdisp2, __float_as_uint(d2));
                if (v2 > 0.f)
                    atomicMax(&ctl->maxv2, __float_as_uint(v2));
                if (a2 > 0.f)
                    atomicMax(&ctl->maxa2, __float_as_uint(a2));
            }
            __syncthreads();                     // (shf and sh serve the next chunk)
        }
    } else {
        // One chunk per block: the block's row of the force kernel's table.
        // This step's potential energy, every step: one partial per warp
        // (written only by active launches, so that an idle one never
        // overwrites partials that still await their sum; the shuffles run in
        // every lane regardless).  Block sums of the maxima every step, of the
        // other reductions on sample steps (their component 0 stays unused).
        double part[kPartF];
        ET<P> eo;
        float d2 = 0.f, v2 = 0.f, a2 = 0.f;
        unsigned int bad = 0u;
        if (sample)
            step_body<P, TPP, true, SM>(a, a.blk_f, blockIdx.x, active, last, pp, spar, part, eo, d2, v2, a2,
                                        bad);
        else
            step_body<P, TPP, false, SM>(a, a.blk_f, blockIdx.x, active, last, pp, spar, part, eo, d2, v2, a2,
                                         bad);
        if (bad)
            atomicOr(&ctl->status, bad);
        store_warp_energy<P>(a, step, a.blk_f[blockIdx.x].w, eo, active);
        block_max3(d2, v2, a2, shf);
        if (sample)
            block_sum<kPartF>(part, sh);
        if (threadIdx.x == 0) {
            const size_t pb = (size_t)a.blk_f[blockIdx.x].w * kPartF;
            if (sample) {
#pragma unroll
                for (int k = 1; k < kPartF; ++k)
                    a.part_f[pb + k] = part[k];
            }
            if (d2 > 0.f)
                atomicMax(&ctl->maxdisp2, __float_as_uint(d2));
            if (v2 > 0.f)
                atomicMax(&ctl->maxv2, __float_as_uint(v2));
            if (a2 > 0.f)
                atomicMax(&ctl->maxa2, __float_as_uint(a2));
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int t = atomicAdd(&ctl->ticket, 1u);
        s_first = (t == 0);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    // The first block to finish adds up the energies of the earlier step that
    // still awaits its sum (the previous step, written by the previous launch):
    // the other blocks are still working, so this is off the critical path.
    if (s_first && pend >= 0)
        finish_epot<P>(a, pend, sh, shf);
    if (!s_last)
        return;

    // ---- last block ----
    __threadfence();
    if (threadIdx.x == 0) {
        s_m[0] = __uint_as_float(atomicExch(&ctl->maxdisp2, 0u));
        s_m[1] = __uint_as_float(atomicExch(&ctl->maxv2, 0u));
        s_m[2] = __uint_as_float(atomicExch(&ctl->maxa2, 0u));
        s_m[3] = ctl->last_maxdisp2;    // displacement of r(step), the positions of this sample
    }
    __syncthreads();
    const unsigned int st = atomicOr(&ctl->status, 0u);
    if (sample && st == 0u)
        finish_reductions<P>(a, IM_LOOP, true, step, s_m[3], sh, shf);   // (its E_pot enters the series)
    if (threadIdx.x == 0) {
        if (sample && st == 0u)
            a.epot_step[step % a.epot_cap] = step;
        // this step's energies: summed into the series here (sample) or by the
        // first block to finish the next launch (or by k_epot_flush)
        ctl->epot_pending = (remaining > 0 && st == 0u && !sample) ? step : -1ll;
        const bool drifted = active && !last;
        unsigned int reb = 0u;
        if (drifted && st == 0u) {
            reb = need_rebuild(a, s_m[0], s_m[1], s_m[2]);
            ctl->step = step + 1;
            ctl->pos_par = pp ^ 1;
            ctl->last_maxdisp2 = s_m[0];
        }
        ctl->rebuild = reb;
        if (sample && st == 0u)
            ctl->obs_count += 1;
        long long rem = remaining;
        if (active)
            rem -= 1;
        ctl->remaining = rem;
        const long long bud = ctl->budget - 1;
        ctl->budget = bud;
        unsigned int s2 = st;
        if (bud <= 0 && rem > 0) {
            atomicOr(&ctl->status, ST_TIMEOUT);
            s2 |= ST_TIMEOUT;
        }
        ctl->ticket = 0u;
        ctl->n_integrate += 1;
        if (a.use_cond) {
            if (a.set_rebuild)
                cudaGraphSetConditional(a.h_rebuild, reb);
            if (a.set_loop)
                cudaGraphSetConditional(a.h_loop, (s2 == 0u && rem > 0) ? 1u : 0u);
        }
        // duration of this launch (one that advanced a step): earliest block start
        // to the end of the last block
        const unsigned long long t0 = ~ctl->t_first_inv;
        const unsigned long long t1 = global_ns();
        if (active) {
            ctl->dev_ns += t1 > t0 ? t1 - t0 : 0ull;
            ctl->dev_launches += 1;
        }
        ctl->t_first_inv = 0ull;
    }
}

// ---------------------------------------------------------------------------
// k_integrate: the per-particle half kick + drift that opens md_step
// (IM_FIRST), and the kinetic reductions alone (IM_SAMPLE, IM_TOTALS, IM_KE).
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kIntBlock) k_integrate(KArgs a)
{
    __shared__ double sh[32 * 12];
    __shared__ float shf[160];
    __shared__ int s_last;
    __shared__ float s_m[3];
    Ctl *ctl = a.ctl;
    const unsigned int st0 = ctl->status;
    const bool halted = st0 != 0u;
    const long long step = ctl->step;
    const int pp = ctl->pos_par, spar = ctl->state_par;
    const int mode = a.imode;
    const bool first = mode == IM_FIRST;
    const bool rec = !first;

    const int4 b = a.blk_i[blockIdx.x];
    const Rep rp = a.rep[b.z];
    const int i = b.x + threadIdx.x;
    const bool valid = (i < b.y) && !halted;
    float d2 = 0.f, v2 = 0.f, a2 = 0.f;
    double kin[4] = {0.0, 0.0, 0.0, 0.0};
    unsigned int bad = 0u;
    if (valid) {
        PState<P> s;
        load_pos<P>(a, pp, i, s);
        load_vel<P>(a, spar, i, s);
        if (rec)
            kinetic<P>(a, s, kin);
        if (first) {
            FT<P> f[3];
            if constexpr (P == FP64) {
                const d4 q = ((const d4 *)a.force)[i];
                f[0] = q.x; f[1] = q.y; f[2] = q.z;
            } else {
                const float4 q = ((const float4 *)a.force)[i];
                f[0] = q.x; f[1] = q.y; f[2] = q.z;
            }
            half_kick<P>(a, s, f[0], f[1], f[2]);
            d2 = drift<P>(a, rp, s, pp ^ 1, spar, i, bad);
            v2 = speed2(s);
            const float im = a.inv_mass[s.sp];
            a2 = __fmul_rn(__fmul_rn(norm2(f[0], f[1], f[2]), im), im);
            store_vel<P>(a, spar, i, s);
        }
    }
    if (bad)
        atomicOr(&ctl->status, bad);
    block_max3(d2, v2, a2, shf);
    if (rec)
        block_sum<4>(kin, sh);
    if (threadIdx.x == 0) {
        if (rec)
#pragma unroll
            for (int k = 0; k < 4; ++k)
                a.part_i[(size_t)blockIdx.x * 4 + k] = kin[k];
        if (d2 > 0.f)
            atomicMax(&ctl->maxdisp2, __float_as_uint(d2));
        if (v2 > 0.f)
            atomicMax(&ctl->maxv2, __float_as_uint(v2));
        if (a2 > 0.f)
            atomicMax(&ctl->maxa2, __float_as_uint(a2));
        __threadfence();
        const unsigned int t = atomicAdd(&ctl->ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();
    if (threadIdx.x == 0) {
        s_m[0] = __uint_as_float(atomicExch(&ctl->maxdisp2, 0u));
        s_m[1] = __uint_as_float(atomicExch(&ctl->maxv2, 0u));
        s_m[2] = __uint_as_float(atomicExch(&ctl->maxa2, 0u));
    }
    __syncthreads();
    const unsigned int st = atomicOr(&ctl->status, 0u);
    if (rec && st == 0u)
        finish_reductions<P>(a, mode, false, step, s_m[0], sh, shf);
    if (threadIdx.x == 0) {
        unsigned int reb = 0u;
        if (first && !halted && st == 0u) {
            reb = need_rebuild(a, s_m[0], s_m[1], s_m[2]);
            ctl->step = step + 1;
            ctl->pos_par = pp ^ 1;
            ctl->last_maxdisp2 = s_m[0];
        }
        if (first)
            ctl->rebuild = reb;
        if (mode == IM_SAMPLE && st == 0u) {
            ctl->obs_count += 1;
            a.epot_step[step % a.epot_cap] = step;
        }
        ctl->ticket = 0u;
        ctl->n_integrate += 1;
        if (a.use_cond && a.set_rebuild)
            cudaGraphSetConditional(a.h_rebuild, reb);
    }
}

// ---------------------------------------------------------------------------
// Cell binning by counting sort (Sec. 2.2: integer cell index per particle,
// particles sorted by cell, start index of each cell) with the cells ordered
// along a space-filling curve (the periodic reorder of Sec. 2.2).
// Kernels: k_bin (cell key + histogram) -> k_scan -> k_scatter ->
// k_permute (deterministic order inside a cell; gather of the state into the
// other buffers) -> k_nbuild (lists from the permuted positions; its last
// block makes the permuted buffers current).  Each returns at once unless a
// rebuild is pending; k_scan clears the histogram for the next binning.
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

// Octant of a coordinate inside its cell (0 or 1 per axis); the three
// interleave into the particle's sub-cell code along a Morton curve, the order
// of the particles inside a cell after each rebuild, so that the particles a
// warp holds are close in space (their neighbours overlap).  (A 4 x 4 x 4
// grid measured 0.25 % slower per MD step.)
__device__ __forceinline__ unsigned int sub2(double x, double cscale, int c)
{
    const int s = (int)floor((x * cscale - (double)c) * 2.0);
    return (unsigned int)(s < 0 ? 0 : (s > 1 ? 1 : s));
}

__device__ __forceinline__ unsigned int sub2f(float x, float cscale, int c)
{
    const int s = (int)floorf((x * cscale - (float)c) * 2.0f);
    return (unsigned int)(s < 0 ? 0 : (s > 1 ? 1 : s));
}

__device__ __forceinline__ int morton6(unsigned int x, unsigned int y, unsigned int z)
{
    return (int)((x & 1u) | ((y & 1u) << 1) | ((z & 1u) << 2) | ((x & 2u) << 2) | ((y & 2u) << 3) |
                 ((z & 2u) << 4));
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
    const int pp = ctl->pos_par;
    int cx, cy, cz, sub;
    if constexpr (P == FP64) {
        const d4 x = ((const d4 *)pos_a(a, pp))[i];
        cx = cell_coord(x.x, rp.cscale, rp.nc);
        cy = cell_coord(x.y, rp.cscale, rp.nc);
        cz = cell_coord(x.z, rp.cscale, rp.nc);
        sub = morton6(sub2(x.x, rp.cscale, cx), sub2(x.y, rp.cscale, cy), sub2(x.z, rp.cscale, cz));
    } else {
        const float4 x = ((const float4 *)pos_a(a, pp))[i];
        cx = cell_coord_f(x.x, rp.cscalef, rp.nc);
        cy = cell_coord_f(x.y, rp.cscalef, rp.nc);
        cz = cell_coord_f(x.z, rp.cscalef, rp.nc);
        sub = morton6(sub2f(x.x, rp.cscalef, cx), sub2f(x.y, rp.cscalef, cy), sub2f(x.z, rp.cscalef, cz));
    }
    const int key = checked(a, a.crank[rp.cell0 + (cz * rp.nc + cy) * rp.nc + cx], a.ncell, 0);
    a.key[i] = key;
    a.skey[i] = sub;
    atomicAdd(&a.ccount[key], 1);
}

// exclusive scan of the cell histogram by one block; also clears the cursors
template <int P>
__global__ void __launch_bounds__(kScanBlock) k_scan(KArgs a)
{
    // Exclusive prefix sum of the cell counts (one block), in tiles of
    // kScanBlock x kScanPer cells: each tile is read and written with coalesced
    // accesses through shared memory, each thread scans kScanPer consecutive
    // counts, and the per-thread sums are scanned across the block.  The
    // counts are cleared for the next binning.
    constexpr int T = kScanBlock, R = kScanPer;
    __shared__ int tile[T * R + T * R / 32];      // padded: one word every 32
    __shared__ int wsum[32];
    __shared__ int s_carry;
    Ctl *ctl = a.ctl;
    if (!rebuild_pending(ctl))
        return;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) {
        atomicAdd((unsigned long long *)&ctl->n_rebuild_k, 1ull);
        s_carry = 0;
    }
    const int n = a.ncell;
    auto at = [](int i) { return i + (i >> 5); };
    for (int base = 0; base < n; base += T * R) {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int i = base + k * T + t;
            tile[at(k * T + t)] = i < n ? a.ccount[i] : 0;
        }
        __syncthreads();
        int v[R], sum = 0;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            v[k] = tile[at(t * R + k)];
            sum += v[k];
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o)
                incl += y;
        }
        if (lane == 31)
            wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            int x = lane < T / 32 ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o)
                    x += y;
            }
            wsum[lane] = x;                       // inclusive sums of the warps
        }
        __syncthreads();
        const int carry = s_carry;
        int run = carry + (w > 0 ? wsum[w - 1] : 0) + incl - sum;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            tile[at(t * R + k)] = run;
            run += v[k];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int i = base + k * T + t;
            if (i < n) {
                a.cstart[i] = tile[at(k * T + t)];
                a.ccount[i] = 0;          // ready for the next binning
                a.ccursor[i] = 0;
            }
        }
        if (t == 0)
            s_carry = carry + wsum[T / 32 - 1];
        __syncthreads();
    }
    if (t == 0)
        a.cstart[n] = s_carry;
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
    const int k = checked(a, a.key[i], a.ncell, 0);
    const int slot = checked(a, a.cstart[k] + atomicAdd(&a.ccursor[k], 1), a.n, 0);
    a.tmpidx[slot] = i;
}

// Final slot of each particle: its cell's start plus the number of particles
// of the same cell that come before it in (sub-cell code, current index)
// order (deterministic), then gather of the whole state into the other
// buffers.
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
    const int pp = ctl->pos_par, spar = ctl->state_par;
    const int i = checked(a, a.tmpidx[s], a.n, 0);
    const int k = checked(a, a.key[i], a.ncell, 0);
    const int b0 = a.cstart[k], b1 = a.cstart[k + 1];
    const int si = a.skey[i];
    int rank = 0;
    for (int t = b0; t < b1; ++t) {
        const int j = checked(a, a.tmpidx[t], a.n, 0);
        const int sj = a.skey[j];
        rank += (sj < si || (sj == si && j < i)) ? 1 : 0;
    }
    const int d = checked(a, b0 + rank, a.n, 0);
    if constexpr (P == FP64) {
        const d4 x = ((const d4 *)pos_a(a, pp))[i];
        ((d4 *)pos_a(a, pp ^ 1))[d] = x;
        ((d4 *)vel_a(a, spar ^ 1))[d] = ((const d4 *)vel_a(a, spar))[i];
        a.rref[d] = make_float4(__double2float_rn(x.x), __double2float_rn(x.y), __double2float_rn(x.z), 0.f);
    } else {
        const float4 x = ((const float4 *)pos_a(a, pp))[i];
        ((float4 *)pos_a(a, pp ^ 1))[d] = x;
        ((float4 *)vel_a(a, spar ^ 1))[d] = ((const float4 *)vel_a(a, spar))[i];
        if constexpr (P == MIXED) {
            ((float4 *)pos_b(a, pp ^ 1))[d] = ((const float4 *)pos_b(a, pp))[i];
            q_of(a, pp ^ 1)[d] = q_of(a, pp)[i];
            ((float4 *)vel_b(a, spar ^ 1))[d] = ((const float4 *)vel_b(a, spar))[i];
        }
        a.rref[d] = make_float4(x.x, x.y, x.z, 0.f);
    }
    img_of(a, spar ^ 1)[d] = img_of(a, spar)[i];
}

// ---------------------------------------------------------------------------
// Neighbour-list build (Sec. 2.2), one warp per cell, one lane per particle
// of the cell (batches of 32).  The warp stages the particles of the 27
// surrounding cells (all cells of the replica when fewer than three fit along
// its edge) in shared memory, in a fixed order (stencil order, then slot order
// inside a cell), dropping those farther than the largest list radius from
// the cell's own box; then every lane tests the staged candidates one after
// the other (each read is a broadcast) against its own particle and appends
// those closer than r_c,ab + skin (plus a rounding margin) to its row of the
// particle-major list nbr[i*Kstride + k], in that order, one store per entry
// kept (the L2 merges the row's words).  No block
// barrier: the cells of a block never wait for one another.  Distances are
// single precision: from the fixed-point copy in MIXED mode, from the
// (rounded) positions otherwise; the list only has to contain every pair
// within r_c + skin, and the margin covers the rounding.  Reads the permuted
// positions (other buffer).  More candidates than fit in shared memory, or
// more particles in the cell than 32, are processed in rounds, so no cell
// size is too large.
// ---------------------------------------------------------------------------
constexpr int kNbStage = 256;    // staged candidates per round and warp

struct NbWarp {
    float4 pos[kNbStage];
    int idx[kNbStage];
    int cell[27];
};

// Position word staged by the neighbour build: MIXED stages the fixed-point copy
// (bits of X, Y, Z, species), whose wrapped differences give the exact minimum
// image; the other modes the single-precision position and species bits.
constexpr bool kNbFixed = true;

template <int P>
__device__ __forceinline__ float4 nb_word(const KArgs &a, int pn, int j)
{
    if constexpr (P == MIXED && kNbFixed) {
        const int4 q = q_of(a, pn)[j];
        return make_float4(__int_as_float(q.x), __int_as_float(q.y), __int_as_float(q.z), __int_as_float(q.w));
    } else if constexpr (P == FP64) {
        const d4 x = ((const d4 *)pos_a(a, pn))[j];
        return make_float4(__double2float_rn(x.x), __double2float_rn(x.y), __double2float_rn(x.z),
                           __int_as_float(species_of(x.w)));
    } else {
        return ((const float4 *)pos_a(a, pn))[j];
    }
}

template <int P>
__device__ __forceinline__ int nb_species(float4 w)
{
    if constexpr (P == MIXED && kNbFixed)
        return __float_as_int(w.w);
    else
        return species_of(w.w);
}

// approximate coordinates of a staged word (for the candidate filter)
template <int P>
__device__ __forceinline__ float3 nb_coords(float4 w, const Rep &rp)
{
    if constexpr (P == MIXED && kNbFixed)
        return make_float3(__uint2float_rn(__float_as_uint(w.x)) * rp.qunit,
                           __uint2float_rn(__float_as_uint(w.y)) * rp.qunit,
                           __uint2float_rn(__float_as_uint(w.z)) * rp.qunit);
    else
        return make_float3(w.x, w.y, w.z);
}

// squared minimum-image distance of two staged words; for the fixed-point
// words in units of the grid (qunit^2), which the caller's radii are scaled to
template <int P>
__device__ __forceinline__ float nb_r2(float4 u, float4 w, const Rep &rp)
{
    float ex, ey, ez;
    if constexpr (P == MIXED && kNbFixed) {
        ex = __int2float_rn((int)(__float_as_uint(u.x) - __float_as_uint(w.x)));
        ey = __int2float_rn((int)(__float_as_uint(u.y) - __float_as_uint(w.y)));
        ez = __int2float_rn((int)(__float_as_uint(u.z) - __float_as_uint(w.z)));
    } else {
        ex = sep_f(u.x, w.x, rp.Lhi, rp.invLf);
        ey = sep_f(u.y, w.y, rp.Lhi, rp.invLf);
        ez = sep_f(u.z, w.z, rp.Lhi, rp.invLf);
    }
    return fmaf(ex, ex, fmaf(ey, ey, ez * ez));
}

// distance of x from the interval [c - h, c + h] on a periodic axis
__device__ __forceinline__ float box_gap(float x, float c, float h, float L, float invL)
{
    return fmaxf(fabsf(sep_f(x, c, L, invL)) - h, 0.0f);
}

// Warp per cell: the lists of the particles of cell c, from the positions in
// buffer pn (the permuted copy being built), by one warp: row i starts at nbr[i * Kstride]
// (the cap) and holds at most K entries (the capacity in use).  Every
// particle's full count is recorded in max_nbr; entries beyond K are dropped
// (the build's last block then grows K and the build is redone).
template <int P>
__device__ __forceinline__ void nbuild_cell_warp(const KArgs &a, int pn, int c, int K, NbWarp &S)
{
    constexpr unsigned FULL = 0xffffffffu;
    Ctl *ctl = a.ctl;
    const int lane = threadIdx.x & 31;
    const int4 cc = a.cxyz[c];
    const Rep rp = a.rep[cc.w];
    const int nc = rp.nc;
    const int nst = nc >= 3 ? 27 : 1;
    const int c0 = a.cstart[c], c1 = a.cstart[c + 1];
    if (c0 == c1)
        return;
    if (lane < nst) {
        int x = cc.x, y = cc.y, z = cc.z;
        if (nst == 27) {
            x = (x + lane % 3 - 1 + nc) % nc;
            y = (y + (lane / 3) % 3 - 1 + nc) % nc;
            z = (z + lane / 9 - 1 + nc) % nc;
        }
        S.cell[lane] = a.crank[rp.cell0 + (z * nc + y) * nc + x];
    }
    __syncwarp();

    // own cell box (centre, half edge) for the candidate filter
    const float edge = rp.Lhi / (float)nc;
    const float hx = 0.5f * edge + 1e-3f;
    const float ccx = ((float)cc.x + 0.5f) * edge, ccy = ((float)cc.y + 0.5f) * edge,
                ccz = ((float)cc.z + 0.5f) * edge;
    const float rlmax2 = fmaxf(fmaxf(a.tab.rl2[0], a.tab.rl2[1]), fmaxf(a.tab.rl2[2], a.tab.rl2[3]));
    const unsigned lt_mask = (1u << lane) - 1u;
    // nb_r2 of the fixed-point words is in units of qunit^2: the list radii follow
    const float r2unit = (P == MIXED && kNbFixed) ? 1.0f / (rp.qunit * rp.qunit) : 1.0f;

    for (int ob = c0; ob < c1; ob += 32) {
        const int i = ob + lane;
        const bool own = i < c1;
        const float4 H = nb_word<P>(a, pn, own ? i : ob);
        const int ti = nb_species<P>(H);
        const float rl0 = own ? a.tab.rl2[ti * 2] * r2unit : -1.0f;      // -1: nothing passes
        const float rl1 = own ? a.tab.rl2[ti * 2 + 1] * r2unit : -1.0f;
        int *row = a.nbr + (size_t)(own ? i : ob) * (size_t)a.Kstride;
        int cnt = 0;          // neighbours found
        int staged = 0;

        // test the staged candidates against the lane's particle, in order; each
        // entry kept goes straight to the lane's row (the L2 merges a row's writes)
        auto scan = [&]() {
            __syncwarp();
#pragma unroll 4
            for (int s = 0; s < staged; ++s) {
                const float4 y = S.pos[s];
                const int jj = S.idx[s];
                const float r2 = nb_r2<P>(H, y, rp);
                const bool in = r2 < (nb_species<P>(y) != 0 ? rl1 : rl0) && jj != i;
                if (in && cnt < K)
                    row[cnt] = jj;
                cnt += in ? 1 : 0;
            }
            __syncwarp();
            staged = 0;
        };

        for (int k = 0; k < nst; ++k) {
            const int cs = a.cstart[S.cell[k]], ce = a.cstart[S.cell[k] + 1];
            for (int t0 = cs; t0 < ce; t0 += 32) {
                if (staged > kNbStage - 32)
                    scan();
                const int t = t0 + lane;
                bool keep = false;
                float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                if (t < ce) {
                    q = nb_word<P>(a, pn, checked(a, t, a.n, 0));
                    keep = true;
                    if (nst == 27) {
                        const float3 x = nb_coords<P>(q, rp);
                        const float gx = box_gap(x.x, ccx, hx, rp.Lhi, rp.invLf);
                        const float gy = box_gap(x.y, ccy, hx, rp.Lhi, rp.invLf);
                        const float gz = box_gap(x.z, ccz, hx, rp.Lhi, rp.invLf);
                        keep = fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < rlmax2;
                    }
                }
                const unsigned m = __ballot_sync(FULL, keep);
                if (keep) {
                    const int sidx = staged + __popc(m & lt_mask);
                    S.pos[sidx] = q;
                    S.idx[sidx] = t;
                }
                staged += __popc(m);
            }
        }
        scan();

        if (own) {
            // padding with the particle itself to a multiple of kUnr entries, so the pair
            // loop reads whole groups without masking
            const int kept = cnt < K ? cnt : K;
            for (int k = kept; k < (kept + kUnr - 1) / kUnr * kUnr && k < K; ++k)
                row[k] = i;
            a.nnbr[i] = kept;
            atomicMax(&ctl->max_nbr, cnt);
        }
        __syncwarp();
    }
}

// Block per cell, for handles with too few cells to occupy the GPU with one
// warp each: the block stages the candidates (kNbCap per round, the same
// order and filter as above), and each of its warps takes kNbPass particles
// of the cell at a time, testing 32 staged candidates per ballot; the list
// rows come out the same as with a warp per cell.
constexpr int kNbCap = 1024;     // staged candidates per round
constexpr int kNbOwn = 256;      // own-cell particles per batch
constexpr int kNbPass = 2;       // own-cell particles tested per warp pass over the candidates

template <int P>
__device__ __forceinline__ void nbuild_cell_block(const KArgs &a, int pn, int c, int K)
{
    __shared__ float4 s_pos[kNbCap];
    __shared__ int s_idx[kNbCap];
    __shared__ int s_cnt[kNbOwn];
    __shared__ int s_pref[28];
    __shared__ int s_cell[27];
    __shared__ int s_wsum[kNbBlockB / 32];

    Ctl *ctl = a.ctl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kNbBlockB / 32;
    const int4 cc = a.cxyz[c];
    const Rep rp = a.rep[cc.w];
    const int nc = rp.nc;
    const int nst = nc >= 3 ? 27 : 1;
    const int c0 = a.cstart[c], c1 = a.cstart[c + 1];
    if (c0 == c1)
        return;

    if (tid < nst) {
        int x = cc.x, y = cc.y, z = cc.z;
        if (nst == 27) {
            x = (x + tid % 3 - 1 + nc) % nc;
            y = (y + (tid / 3) % 3 - 1 + nc) % nc;
            z = (z + tid / 9 - 1 + nc) % nc;
        }
        s_cell[tid] = a.crank[rp.cell0 + (z * nc + y) * nc + x];
    }
    __syncthreads();
    if (tid == 0) {
        int s = 0;
        for (int k = 0; k < nst; ++k) {
            s_pref[k] = s;
            s += a.cstart[s_cell[k] + 1] - a.cstart[s_cell[k]];
        }
        s_pref[nst] = s;
    }
    __syncthreads();
    const int total = s_pref[nst];

    // own cell box (centre, half edge) for the candidate filter
    const float edge = rp.Lhi / (float)nc;
    const float hx = 0.5f * edge + 1e-3f;
    const float ccx = ((float)cc.x + 0.5f) * edge, ccy = ((float)cc.y + 0.5f) * edge,
                ccz = ((float)cc.z + 0.5f) * edge;
    const float rlmax2 = fmaxf(fmaxf(a.tab.rl2[0], a.tab.rl2[1]), fmaxf(a.tab.rl2[2], a.tab.rl2[3]));
    const unsigned lt_mask = (1u << lane) - 1u;
    // nb_r2 of the fixed-point words is in units of qunit^2: the list radii follow
    const float r2unit = (P == MIXED && kNbFixed) ? 1.0f / (rp.qunit * rp.qunit) : 1.0f;

    for (int ob = c0; ob < c1; ob += kNbOwn) {
        const int nown = min(kNbOwn, c1 - ob);
        for (int t = tid; t < nown; t += kNbBlockB)
            s_cnt[t] = 0;
        int staged = 0;
        for (int base = 0; base < total; base += kNbBlockB) {
            // stage candidates base .. base + kNbBlockB - 1, order-preserving compaction
            const int t = base + tid;
            bool keep = false;
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            int j = 0;
            if (t < total) {
                int k = 0;
                while (k + 1 < nst && s_pref[k + 1] <= t)
                    ++k;
                j = checked(a, a.cstart[s_cell[k]] + (t - s_pref[k]), a.n, 0);
                q = nb_word<P>(a, pn, j);
                keep = true;
                if (nst == 27) {
                    const float3 x = nb_coords<P>(q, rp);
                    const float gx = box_gap(x.x, ccx, hx, rp.Lhi, rp.invLf);
                    const float gy = box_gap(x.y, ccy, hx, rp.Lhi, rp.invLf);
                    const float gz = box_gap(x.z, ccz, hx, rp.Lhi, rp.invLf);
                    keep = fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < rlmax2;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (lane == 0)
                s_wsum[warp] = __popc(m);
            __syncthreads();
            int off = staged, add = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                off += (w < warp) ? s_wsum[w] : 0;
                add += s_wsum[w];
            }
            if (keep) {
                const int s = off + __popc(m & lt_mask);
                s_pos[s] = q;
                s_idx[s] = j;
            }
            staged += add;
            __syncthreads();
            if (staged <= kNbCap - kNbBlockB && base + kNbBlockB < total)
                continue;

            // scan the staged candidates: each warp pass takes kNbPass particles of
            // the batch, so that every staged candidate read serves kNbPass tests
            for (int o0 = warp * kNbPass; o0 < nown; o0 += NW * kNbPass) {
                float4 H[kNbPass];
                float rl0[kNbPass], rl1[kNbPass];
                int cnt[kNbPass];
#pragma unroll
                for (int p = 0; p < kNbPass; ++p) {
                    const bool ok = o0 + p < nown;
                    H[p] = nb_word<P>(a, pn, ob + (ok ? o0 + p : 0));
                    const int ti = nb_species<P>(H[p]);
                    rl0[p] = ok ? a.tab.rl2[ti * 2] * r2unit : -1.0f;       // -1: nothing passes
                    rl1[p] = ok ? a.tab.rl2[ti * 2 + 1] * r2unit : -1.0f;
                    cnt[p] = ok ? s_cnt[o0 + p] : 0;
                }
                for (int s0 = 0; s0 < staged; s0 += 32) {
                    const int s = s0 + lane;
                    const bool sv = s < staged;
                    const float4 y = sv ? s_pos[s] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const int jj = sv ? s_idx[s] : -1;
                    const bool tj = nb_species<P>(y) != 0;
#pragma unroll
                    for (int p = 0; p < kNbPass; ++p) {
                        const int i = ob + o0 + p;
                        const float r2 = nb_r2<P>(H[p], y, rp);
                        const bool in = sv && jj != i && r2 < (tj ? rl1[p] : rl0[p]);
                        const unsigned mm = __ballot_sync(0xffffffffu, in);
                        const int at = cnt[p] + __popc(mm & lt_mask);
                        if (in && at < K)
                            a.nbr[(size_t)i * (size_t)a.Kstride + at] = jj;
                        cnt[p] += __popc(mm);
                    }
                }
                if (lane == 0)
#pragma unroll
                    for (int p = 0; p < kNbPass; ++p)
                        if (o0 + p < nown)
                            s_cnt[o0 + p] = cnt[p];
            }
            staged = 0;
            __syncthreads();
        }
        for (int o = tid; o < nown; o += kNbBlockB) {
            const int cnt = s_cnt[o];
            a.nnbr[ob + o] = cnt < K ? cnt : K;
            // pad the row with the particle itself to a multiple of kUnr entries, so the
            // pair loop reads whole groups without masking (K is a multiple of 8)
            for (int k = cnt; k < (cnt + kUnr - 1) / kUnr * kUnr && k < K; ++k)
                a.nbr[(size_t)(ob + o) * (size_t)a.Kstride + k] = ob + o;
            atomicMax(&ctl->max_nbr, cnt);
        }
        __syncthreads();
    }
}

// List capacity after a build whose longest list held mx > K entries (the
// fixed-size list of Sec. 2.2 grown in place): a quarter more than needed,
// rounded up to whole groups of 8, at most the cap Kmax (a multiple of 8, so
// the result still holds mx entries whenever mx <= Kmax).
__device__ __forceinline__ int grown_capacity(int mx, int Kmax)
{
    const int want = (mx + (mx + 3) / 4 + 7) / 8 * 8;
    return want < Kmax ? want : Kmax;
}

// The neighbour build closes the rebuild chain.  The last block to finish
// (ticket pattern) reads the longest list of the build and
//   - makes the permuted buffers current if every list fitted its K entries;
//   - otherwise, if the longest list fits the cap, raises K (grown_capacity)
//     and asks for the build to be redone (Ctl::regrow, and the graph's regrow
//     condition): the redo (nb_retry = 1, same positions, so the same counts)
//     then fits, and its last block makes the buffers current;
//   - otherwise reports ST_OVERFLOW, leaving the buffers of the last completed
//     step current.
// The pending check is read once per block (the status can change during the
// launch) and every block takes a ticket.  k_nbuild: warp w of block b takes
// cells kNbCells b + w, then kNbCells gridDim.x further on, ...; k_nbuild_blk:
// block b takes cells b, b + gridDim.x, ...

// First thread of every block of the build: is a build (or its redo) pending,
// and the capacity in use; counts the launch.
__device__ __forceinline__ void nbuild_begin(const KArgs &a, int &s_go, int &s_K)
{
    Ctl *ctl = a.ctl;
    if (threadIdx.x == 0) {
        s_go = (rebuild_pending(ctl) && (a.nb_retry == 0 || ctl->regrow != 0u)) ? 1 : 0;
        s_K = ctl->K;
        if (s_go && blockIdx.x == 0) {
            atomicAdd((unsigned long long *)&ctl->n_rebuild_k, 1ull);
            if (a.nb_retry)
                atomicAdd((unsigned long long *)&ctl->regrows, 1ull);
            else
                atomicAdd((unsigned long long *)&ctl->rebuilds, 1ull);
        }
    }
}

// Every block's ticket; the last block swaps in the permuted buffers, grows the
// capacity and asks for the redo, or reports the overflow (see above).
__device__ __forceinline__ void nbuild_end(const KArgs &a, int s_go, int s_K)
{
    Ctl *ctl = a.ctl;
    if (threadIdx.x == 0) {
        __threadfence();                    // this block's list counts before its ticket
        const unsigned int t = atomicAdd(&ctl->ticket, 1u);
        if (t == gridDim.x - 1) {
            __threadfence();
            unsigned int regrow = 0u;
            if (s_go && atomicOr(&ctl->status, 0u) == 0u) {
                const int mx = atomicMax(&ctl->max_nbr, 0);
                if (mx <= s_K) {
                    ctl->pos_par ^= 1;
                    ctl->state_par ^= 1;
                    ctl->last_maxdisp2 = 0.f;   // the lists start from these positions
                } else if (mx <= ctl->Kmax && a.nb_retry == 0) {
                    ctl->K = grown_capacity(mx, ctl->Kmax);
                    regrow = 1u;
                } else {
                    atomicOr(&ctl->status, ST_OVERFLOW);
                }
            }
            if (s_go || a.nb_retry == 0)
                ctl->regrow = regrow;
            ctl->ticket = 0u;
            if (a.use_cond && a.set_regrow)
                cudaGraphSetConditional(a.h_regrow, regrow);
        }
    }
}

template <int P>
__global__ void __launch_bounds__(kNbBlock) k_nbuild(KArgs a)
{
    __shared__ NbWarp s_nb[kNbCells];
    __shared__ int s_go, s_K;
    nbuild_begin(a, s_go, s_K);
    __syncthreads();
    if (s_go) {
        const int pn = a.ctl->pos_par ^ 1;
        const int w = threadIdx.x >> 5;
        for (int c = blockIdx.x * kNbCells + w; c < a.ncell; c += gridDim.x * kNbCells)
            nbuild_cell_warp<P>(a, pn, c, s_K, s_nb[w]);
    }
    __syncthreads();
    nbuild_end(a, s_go, s_K);
}

template <int P>
__global__ void __launch_bounds__(kNbBlockB) k_nbuild_blk(KArgs a)
{
    __shared__ int s_go, s_K;
    nbuild_begin(a, s_go, s_K);
    __syncthreads();
    if (s_go) {
        const int pn = a.ctl->pos_par ^ 1;
        for (int c = blockIdx.x; c < a.ncell; c += gridDim.x)
            nbuild_cell_block<P>(a, pn, c, s_K);
    }
    __syncthreads();
    nbuild_end(a, s_go, s_K);
}

template <int P>
__global__ void __launch_bounds__(kIntBlock) k_load(KArgs a)
{
    Ctl *ctl = a.ctl;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->rebuild = 1u;
        atomicAdd((unsigned long long *)&ctl->n_other, 1ull);
    }
    const int4 b = a.blk_i[blockIdx.x];
    const int i = b.x + threadIdx.x;
    if (i >= b.y)
        return;
    const int pp = ctl->pos_par, spar = ctl->state_par;
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
        ((d4 *)pos_a(a, pp))[i] = p;
        ((d4 *)vel_a(a, spar))[i] = v;
    } else if constexpr (P == MIXED) {
        float H[3], l[3];
        for (int k = 0; k < 3; ++k) {
            // high word on the grid: multiples of rp.grid are exact in float for |x| < 2L
            const double h = rint(x[k] * (double)rp.inv_grid) * (double)rp.grid;
            H[k] = (float)h;
            l[k] = __double2float_rn(x[k] - h);
        }
        ((float4 *)pos_a(a, pp))[i] = make_float4(H[0], H[1], H[2], __int_as_float(sp));
        ((float4 *)pos_b(a, pp))[i] = make_float4(l[0], l[1], l[2], 0.f);
        q_of(a, pp)[i] = make_int4((int)fixq(H[0], l[0], rp), (int)fixq(H[1], l[1], rp),
                                   (int)fixq(H[2], l[2], rp), sp);
        ds vx = ds_from_double(vv[0]), vy = ds_from_double(vv[1]), vz = ds_from_double(vv[2]);
        ((float4 *)vel_a(a, spar))[i] = make_float4(vx.hi, vy.hi, vz.hi, 0.f);
        ((float4 *)vel_b(a, spar))[i] = make_float4(vx.lo, vy.lo, vz.lo, 0.f);
    } else {
        float fx = __double2float_rn(x[0]), fy = __double2float_rn(x[1]), fz = __double2float_rn(x[2]);
        const float L = rp.Lhi;
        // a coordinate just below L can round to L: it is 0 of the next image
        if (fx >= L) { fx = 0.f; im[0] += 1; }
        if (fy >= L) { fy = 0.f; im[1] += 1; }
        if (fz >= L) { fz = 0.f; im[2] += 1; }
        ((float4 *)pos_a(a, pp))[i] = make_float4(fx, fy, fz, __int_as_float(sp));
        ((float4 *)vel_a(a, spar))[i] = make_float4((float)vv[0], (float)vv[1], (float)vv[2], 0.f);
    }
    img_of(a, spar)[i] = make_int4(im[0], im[1], im[2], i);
}

// Write the state back to the staging area in the original order.
template <int P>
__global__ void __launch_bounds__(kIntBlock) k_getstate(KArgs a)
{
    const Ctl *ctl = a.ctl;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd((unsigned long long *)&a.ctl->n_other, 1ull);
    if (s >= a.n)
        return;
    const int pp = ctl->pos_par, spar = ctl->state_par;
    const int4 im = img_of(a, spar)[s];
    const size_t t = (size_t)im.w;
    double x[3], v[3];
    if constexpr (P == FP64) {
        const d4 p = ((const d4 *)pos_a(a, pp))[s], w = ((const d4 *)vel_a(a, spar))[s];
        x[0] = p.x; x[1] = p.y; x[2] = p.z;
        v[0] = w.x; v[1] = w.y; v[2] = w.z;
    } else if constexpr (P == MIXED) {
        const float4 H = ((const float4 *)pos_a(a, pp))[s], l = ((const float4 *)pos_b(a, pp))[s];
        const float4 vh = ((const float4 *)vel_a(a, spar))[s], vl = ((const float4 *)vel_b(a, spar))[s];
        x[0] = (double)H.x + (double)l.x; x[1] = (double)H.y + (double)l.y; x[2] = (double)H.z + (double)l.z;
        v[0] = (double)vh.x + (double)vl.x; v[1] = (double)vh.y + (double)vl.y; v[2] = (double)vh.z + (double)vl.z;
    } else {
        const float4 p = ((const float4 *)pos_a(a, pp))[s], w = ((const float4 *)vel_a(a, spar))[s];
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
    const Ctl *ctl = a.ctl;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd((unsigned long long *)&a.ctl->n_other, 1ull);
    if (s >= a.n)
        return;
    const size_t t = (size_t)img_of(a, ctl->state_par)[s].w;
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
    const Ctl *ctl = a.ctl;
    if (ctl->status)
        return;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd((unsigned long long *)&a.ctl->n_other, 1ull);
    const int4 b = a.blk_i[blockIdx.x];
    const int i = b.x + threadIdx.x;
    if (i >= b.y)
        return;
    const int spar = ctl->state_par;
    const double f = a.scale[b.z];
    if constexpr (P == FP64) {
        d4 v = ((d4 *)vel_a(a, spar))[i];
        v.x *= f; v.y *= f; v.z *= f;
        ((d4 *)vel_a(a, spar))[i] = v;
    } else if constexpr (P == MIXED) {
        const ds fs = ds_from_double(f);
        float4 vh = ((float4 *)vel_a(a, spar))[i], vl = ((float4 *)vel_b(a, spar))[i];
        ds x = ds_mul(ds_from(vh.x, vl.x), fs), y = ds_mul(ds_from(vh.y, vl.y), fs),
           z = ds_mul(ds_from(vh.z, vl.z), fs);
        ((float4 *)vel_a(a, spar))[i] = make_float4(x.hi, y.hi, z.hi, 0.f);
        ((float4 *)vel_b(a, spar))[i] = make_float4(x.lo, y.lo, z.lo, 0.f);
    } else {
        float4 v = ((float4 *)vel_a(a, spar))[i];
        const float ff = (float)f;
        v.x *= ff; v.y *= ff; v.z *= ff;
        ((float4 *)vel_a(a, spar))[i] = v;
    }
}

template <int P>
__global__ void k_set_steps(KArgs a)
{
    a.ctl->remaining = a.nsteps;
    a.ctl->budget = a.budget > 0 ? a.budget : a.nsteps + 64;
    a.ctl->n_other += 1;
}

// clear a reported status so that the handle can be inspected and reused
template <int P>
__global__ void k_reset(KArgs a)
{
    a.ctl->status = 0u;
    a.ctl->ticket = 0u;
    a.ctl->maxdisp2 = 0u;
    a.ctl->maxv2 = 0u;
    a.ctl->maxa2 = 0u;
    a.ctl->remaining = 0;
    a.ctl->n_other += 1;
}

// ---------------------------------------------------------------------------
// Andersen heat bath (Sec. 2.3): every particle draws a Maxwell-Boltzmann
// velocity from the rand48 sequence (x_{n+1} = a x_n + c mod 2^48; deviate n is
// x_{n+1} / 2^48).  Particle i (original index) is thread i of a leapfrog over
// the n particles: collision e uses its deviates (4e + k) n + i, k = 0..3.
// The first is reached by jumping ahead (the affine map raised to a power by
// squaring, exact in 64-bit integer arithmetic modulo 2^48), the others by the
// leapfrog x -> A_n x + C_n.  Box-Muller turns them into three normals; then
// k_andersen_fix removes the mean velocity and rescales to the target
// temperature exactly, per replica, from the FP64 totals.
// ---------------------------------------------------------------------------
constexpr unsigned long long kR48A = 0x5DEECE66DULL, kR48C = 0xBULL, kR48Mask = 0xFFFFFFFFFFFFULL;

__device__ __forceinline__ unsigned long long r48_jump(unsigned long long x, unsigned long long p)
{
    unsigned long long A = 1, C = 0, Ab = kR48A, Cb = kR48C;   // result map, map^(2^k)
    while (p) {
        if (p & 1ull) {
            A = (Ab * A) & kR48Mask;
            C = (Ab * C + Cb) & kR48Mask;
        }
        Cb = (Ab * Cb + Cb) & kR48Mask;
        Ab = (Ab * Ab) & kR48Mask;
        p >>= 1;
    }
    return (A * x + C) & kR48Mask;
}

template <int P>
__global__ void __launch_bounds__(kIntBlock) k_andersen(KArgs a)
{
    const Ctl *ctl = a.ctl;
    if (ctl->status)
        return;
    const int4 b = a.blk_i[blockIdx.x];
    const int i = b.x + threadIdx.x;
    if (i >= b.y)
        return;
    const int spar = ctl->state_par;
    const int orig = img_of(a, spar)[i].w;
    int sp;
    if constexpr (P == FP64)
        sp = species_of(((const d4 *)pos_a(a, ctl->pos_par))[i].w);
    else
        sp = species_of(((const float4 *)pos_a(a, ctl->pos_par))[i].w);
    unsigned long long x = r48_jump(a.r48_x0, (unsigned long long)a.r48_base + (unsigned long long)orig + 1ull);
    double u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        u[k] = (double)x * 0x1p-48;
        x = (a.r48_AN * x + a.r48_CN) & kR48Mask;
    }
    const double s = sqrt(a.scale[b.z] / a.mass[sp]);
    const double r1 = s * sqrt(-2.0 * log(1.0 - u[0])), r2 = s * sqrt(-2.0 * log(1.0 - u[2]));
    double s1, c1, s3, c3;
    sincospi(2.0 * u[1], &s1, &c1);
    sincospi(2.0 * u[3], &s3, &c3);
    const double v[3] = {r1 * c1, r1 * s1, r2 * c3};
    if constexpr (P == FP64) {
        d4 w;
        w.x = v[0]; w.y = v[1]; w.z = v[2]; w.w = 0.0;
        ((d4 *)vel_a(a, spar))[i] = w;
    } else if constexpr (P == MIXED) {
        const ds x0 = ds_from_double(v[0]), y0 = ds_from_double(v[1]), z0 = ds_from_double(v[2]);
        ((float4 *)vel_a(a, spar))[i] = make_float4(x0.hi, y0.hi, z0.hi, 0.f);
        ((float4 *)vel_b(a, spar))[i] = make_float4(x0.lo, y0.lo, z0.lo, 0.f);
    } else {
        ((float4 *)vel_a(a, spar))[i] = make_float4((float)v[0], (float)v[1], (float)v[2], 0.f);
    }
}

// v <- (v - P/M) s with s = sqrt(T (3N - 3) / (2 E_kin')), E_kin' = E_kin - |P|^2 / 2M,
// from the per-replica totals (E_kin, P) of the drawn velocities
template <int P>
__global__ void __launch_bounds__(kIntBlock) k_andersen_fix(KArgs a)
{
    const Ctl *ctl = a.ctl;
    if (ctl->status)
        return;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd((unsigned long long *)&a.ctl->n_other, 1ull);
    const int4 b = a.blk_i[blockIdx.x];
    const int i = b.x + threadIdx.x;
    if (i >= b.y)
        return;
    const Rep &rp = a.rep[b.z];
    const Obs &t = a.totals[b.z];
    const double M = rp.mtot;
    const double cx = t.p[0] / M, cy = t.p[1] / M, cz = t.p[2] / M;
    const double ek = t.e_kin - 0.5 * (t.p[0] * t.p[0] + t.p[1] * t.p[1] + t.p[2] * t.p[2]) / M;
    const double T = a.scale[b.z];
    const double f = (rp.n > 1 && T > 0.0 && ek > 0.0) ? sqrt(T * (3.0 * rp.n - 3.0) / (2.0 * ek)) : 0.0;
    const int spar = ctl->state_par;
    if constexpr (P == FP64) {
        d4 v = ((d4 *)vel_a(a, spar))[i];
        v.x = (v.x - cx) * f; v.y = (v.y - cy) * f; v.z = (v.z - cz) * f;
        ((d4 *)vel_a(a, spar))[i] = v;
    } else if constexpr (P == MIXED) {
        const float4 vh = ((float4 *)vel_a(a, spar))[i], vl = ((float4 *)vel_b(a, spar))[i];
        const ds x = ds_from_double((ds_to_double(ds_from(vh.x, vl.x)) - cx) * f);
        const ds y = ds_from_double((ds_to_double(ds_from(vh.y, vl.y)) - cy) * f);
        const ds z = ds_from_double((ds_to_double(ds_from(vh.z, vl.z)) - cz) * f);
        ((float4 *)vel_a(a, spar))[i] = make_float4(x.hi, y.hi, z.hi, 0.f);
        ((float4 *)vel_b(a, spar))[i] = make_float4(x.lo, y.lo, z.lo, 0.f);
    } else {
        float4 v = ((float4 *)vel_a(a, spar))[i];
        v.x = (float)((v.x - cx) * f); v.y = (float)((v.y - cy) * f); v.z = (float)((v.z - cz) * f);
        ((float4 *)vel_a(a, spar))[i] = v;
    }
}

// Snapshot for the time-correlation functions (Sec. 2.5): unwrapped positions
// r + L n (FP64) and species, stored by original particle index.
template <int P>
__global__ void __launch_bounds__(kIntBlock) k_snapshot(KArgs a)
{
    const Ctl *ctl = a.ctl;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd((unsigned long long *)&a.ctl->n_other, 1ull);
    const int4 b = a.blk_i[blockIdx.x];
    const int i = b.x + threadIdx.x;
    if (i >= b.y)
        return;
    const double L = a.rep[b.z].L;
    const int pp = ctl->pos_par, spar = ctl->state_par;
    const int4 im = img_of(a, spar)[i];
    double x[3];
    int sp;
    if constexpr (P == FP64) {
        const d4 p = ((const d4 *)pos_a(a, pp))[i];
        x[0] = p.x; x[1] = p.y; x[2] = p.z;
        sp = species_of(p.w);
    } else if constexpr (P == MIXED) {
        const float4 H = ((const float4 *)pos_a(a, pp))[i], l = ((const float4 *)pos_b(a, pp))[i];
        x[0] = (double)H.x + (double)l.x; x[1] = (double)H.y + (double)l.y; x[2] = (double)H.z + (double)l.z;
        sp = species_of(H.w);
    } else {
        const float4 p = ((const float4 *)pos_a(a, pp))[i];
        x[0] = p.x; x[1] = p.y; x[2] = p.z;
        sp = species_of(p.w);
    }
    const size_t t = (size_t)im.w;
    a.snap[3 * t + 0] = __dadd_rn(x[0], __dmul_rn(L, (double)im.x));
    a.snap[3 * t + 1] = __dadd_rn(x[1], __dmul_rn(L, (double)im.y));
    a.snap[3 * t + 2] = __dadd_rn(x[2], __dmul_rn(L, (double)im.z));
    a.snap_species[t] = sp;
}

// Sum the energies of a step that still awaits it into the per-step series
// (before the host reads the series, and before a force evaluation outside
// the step loop reuses the partials).  One block.
template <int P>
__global__ void __launch_bounds__(kForceBlock) k_epot_flush(KArgs a)
{
    __shared__ double sh[32 * kPartF];
    __shared__ float shf[160];
    const long long pend = a.ctl->epot_pending;
    if (pend >= 0)
        finish_epot<P>(a, pend, sh, shf);
    __syncthreads();
    if (threadIdx.x == 0) {
        a.ctl->epot_pending = -1;
        a.ctl->n_other += 1;
    }
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
    k.force[0][0] = (const void *)k_force<P, 1, false>;
    k.force[0][1] = (const void *)k_force<P, 2, false>;
    k.force[0][2] = (const void *)k_force<P, 4, false>;
    k.force[0][3] = (const void *)k_force<P, 8, false>;
    k.force[0][4] = (const void *)k_force<P, 16, false>;
    k.force[0][5] = (const void *)k_force<P, 32, false>;
    k.step[0][0] = (const void *)k_step<P, 1, false, false>;
    k.step[0][1] = (const void *)k_step<P, 2, false, false>;
    k.step[0][2] = (const void *)k_step<P, 4, false, false>;
    k.step[0][3] = (const void *)k_step<P, 8, false, false>;
    k.step[0][4] = (const void *)k_step<P, 16, false, false>;
    k.step[0][5] = (const void *)k_step<P, 32, false, false>;
    // smoothed potential (Sec. 4): the common lane counts only
    k.force[1][0] = (const void *)k_force<P, 1, true>;
    k.force[1][1] = (const void *)k_force<P, 2, true>;
    k.force[1][2] = (const void *)k_force<P, 4, true>;
    k.force[1][3] = (const void *)k_force<P, 8, true>;
    k.force[1][4] = nullptr;
    k.force[1][5] = nullptr;
    k.step[1][0] = (const void *)k_step<P, 1, true, false>;
    k.step[1][1] = (const void *)k_step<P, 2, true, false>;
    k.step[1][2] = (const void *)k_step<P, 4, true, false>;
    k.step[1][3] = (const void *)k_step<P, 8, true, false>;
    k.step[1][4] = nullptr;
    k.step[1][5] = nullptr;
    // resident blocks sweeping runs of chunks: single-precision pair loops at 1 and 2 lanes
    // (at 4 lanes the chunk loop costs registers and was measured slower)
    for (int m = 0; m < 2; ++m)
        for (int l = 0; l < 2; ++l)
            k.step_sweep[m][l] = nullptr;
    if constexpr (P != FP64) {
        k.step_sweep[0][0] = (const void *)k_step<P, 1, false, true>;
        k.step_sweep[0][1] = (const void *)k_step<P, 2, false, true>;
        k.step_sweep[1][0] = (const void *)k_step<P, 1, true, true>;
        k.step_sweep[1][1] = (const void *)k_step<P, 2, true, true>;
    }
    k.bin = (const void *)k_bin<P>;
    k.scan = (const void *)k_scan<P>;
    k.scatter = (const void *)k_scatter<P>;
    k.permute = (const void *)k_permute<P>;
    k.nbuild = (const void *)k_nbuild<P>;
    k.nbuild_blk = (const void *)k_nbuild_blk<P>;
    k.load = (const void *)k_load<P>;
    k.getstate = (const void *)k_getstate<P>;
    k.expforce = (const void *)k_expforce<P>;
    k.scale = (const void *)k_scale<P>;
    k.set_steps = (const void *)k_set_steps<P>;
    k.reset = (const void *)k_reset<P>;
    k.mark_rebuild = (const void *)k_mark_rebuild<P>;
    k.epot_flush = (const void *)k_epot_flush<P>;
    k.andersen = (const void *)k_andersen<P>;
    k.andersen_fix = (const void *)k_andersen_fix<P>;
    k.snapshot = (const void *)k_snapshot<P>;
    return k;
}

}  // namespace mdk
