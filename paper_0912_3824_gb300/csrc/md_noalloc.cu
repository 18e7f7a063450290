// md_noalloc.cu -- force evaluation that allocates no device memory.
//
// Some callers cannot allocate device memory at the moment they need forces:
// an out-of-memory handler that must still evaluate a configuration after an
// allocation has failed, a host application whose memory manager owns the
// whole device and forbids cudaMalloc / cudaFree outside its own pool, or
// code that is certified to allocate nothing after start-up.  For them,
// md_forces_noalloc() evaluates forces, per-particle energies and the
// energy / virial totals of one periodic configuration by a direct sum over
// all pairs, using only the caller's input and output arrays plus a fixed
// scratch area that lives in this library's own device memory.
//
// That scratch is a file-scope __device__ array, reserved on every GPU that
// loads the library for the life of the process.  Host code cannot pass the
// array's name to a kernel (on the host it only names a stand-in), so its
// device address is looked up once per device with cudaGetSymbolAddress().
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdio>
#include <mutex>

#include "md.h"

namespace {

constexpr int kBlock = 128;
constexpr int kMaxBlocks = 8192;   // n <= kMaxBlocks * kBlock = MD_NOALLOC_MAX_N
constexpr int kPart = 8;           // e_pot, virial, w_xx, w_yy, w_zz, w_xy, w_xz, w_yz
constexpr int kMaxDevices = 64;

static_assert((long long)kMaxBlocks * kBlock == MD_NOALLOC_MAX_N, "scratch sized for MD_NOALLOC_MAX_N");

// Per-block partial sums, the ticket that elects the block finishing the
// totals, and a flag raised by any block that met a species outside
// [0, n_species) (512 KiB + 256 B).  ticket and bad are cleared by every call.
struct Scratch {
    double part[kMaxBlocks * kPart];
    unsigned int ticket;
    unsigned int bad;
    unsigned int pad[62];
};

static __device__ __align__(256) Scratch g_noalloc_scratch;

struct Pot {
    double rc2[4], sig2[4], eps4[4], eps48[4], shift[4];
};

__device__ __forceinline__ double min_image(double d, double L, double invL)
{
    return d - L * rint(d * invL);
}

// Species code of a particle, clamped into [0, nsp) so that it always indexes
// the pair table; an out-of-range code raises the call's bad flag.
__device__ __forceinline__ int species_in_range(int t, int nsp, Scratch *s)
{
    if (t < 0 || t >= nsp) {
        atomicOr(&s->bad, 1u);
        return t < 0 ? 0 : nsp - 1;
    }
    return t;
}

// One thread per particle i, looping over every j through shared-memory tiles
// of positions; pair arithmetic in double (FP64 mode) or single precision on
// separations formed in double (the other modes).
template <bool FP64MATH>
__global__ void __launch_bounds__(kBlock) k_forces_allpairs(Pot pot, int n, int nsp, double L, const int *species,
                                                            const double *pos, double *force, double *energy,
                                                            double *totals, Scratch *s)
{
    __shared__ double tx[kBlock], ty[kBlock], tz[kBlock];
    __shared__ int tt[kBlock];
    __shared__ double red[kBlock / 32][kPart];
    __shared__ int is_last;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    const double invL = 1.0 / L;
    double xi = 0.0, yi = 0.0, zi = 0.0;
    int ti = 0;
    bool ti_bad = false;
    if (i < n) {
        xi = pos[3 * (size_t)i];
        yi = pos[3 * (size_t)i + 1];
        zi = pos[3 * (size_t)i + 2];
        ti_bad = species[i] < 0 || species[i] >= nsp;
        ti = species_in_range(species[i], nsp, s);
    }
    double fx = 0.0, fy = 0.0, fz = 0.0, acc[kPart] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int j0 = 0; j0 < n; j0 += kBlock) {
        const int j = j0 + threadIdx.x;
        if (j < n) {
            tx[threadIdx.x] = pos[3 * (size_t)j];
            ty[threadIdx.x] = pos[3 * (size_t)j + 1];
            tz[threadIdx.x] = pos[3 * (size_t)j + 2];
            tt[threadIdx.x] = species_in_range(species[j], nsp, s);
        }
        __syncthreads();
        const int m = min(kBlock, n - j0);
        if (i < n) {
            for (int k = 0; k < m; ++k) {
                if (j0 + k == i)
                    continue;
                const double dx = min_image(xi - tx[k], L, invL);
                const double dy = min_image(yi - ty[k], L, invL);
                const double dz = min_image(zi - tz[k], L, invL);
                const double r2 = dx * dx + dy * dy + dz * dz;
                const int ab = ti * 2 + tt[k];
                if (!(r2 < pot.rc2[ab]))
                    continue;
                double fr, v;
                if (FP64MATH) {
                    const double ir2 = 1.0 / r2;
                    const double s2 = pot.sig2[ab] * ir2;
                    const double s6 = s2 * s2 * s2;
                    fr = pot.eps48[ab] * ir2 * s6 * (s6 - 0.5);
                    v = pot.eps4[ab] * s6 * (s6 - 1.0) - pot.shift[ab];
                } else {
                    const float ir2 = 1.0f / (float)r2;
                    const float s2 = (float)pot.sig2[ab] * ir2;
                    const float s6 = s2 * s2 * s2;
                    fr = (double)((float)pot.eps48[ab] * ir2 * s6 * (s6 - 0.5f));
                    v = (double)((float)pot.eps4[ab] * s6 * (s6 - 1.0f) - (float)pot.shift[ab]);
                }
                fx += fr * dx;
                fy += fr * dy;
                fz += fr * dz;
                acc[0] += v;
                acc[1] += fr * r2;
                acc[2] += fr * dx * dx;
                acc[3] += fr * dy * dy;
                acc[4] += fr * dz * dz;
                acc[5] += fr * dx * dy;
                acc[6] += fr * dx * dz;
                acc[7] += fr * dy * dz;
            }
        }
        __syncthreads();
    }
    if (i < n) {
        const double poison = ti_bad ? __longlong_as_double(0x7ff8000000000000ll) : 0.0;   // NaN
        force[3 * (size_t)i] = fx + poison;
        force[3 * (size_t)i + 1] = fy + poison;
        force[3 * (size_t)i + 2] = fz + poison;
        if (energy)
            energy[i] = 0.5 * acc[0] + poison;
    }
    // block sums in a fixed order, then the last block adds the blocks' sums
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kPart; ++k) {
        double v = 0.5 * acc[k];
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0)
            red[w][k] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < kPart; ++k) {
            double v = 0.0;
            for (int q = 0; q < kBlock / 32; ++q)
                v += red[q][k];
            s->part[(size_t)blockIdx.x * kPart + k] = v;
        }
        __threadfence();
        is_last = atomicAdd(&s->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last)
        return;
    __threadfence();
    if (threadIdx.x < kPart) {
        double v = 0.0;
        for (unsigned int b = 0; b < gridDim.x; ++b)
            v += ((volatile double *)s->part)[(size_t)b * kPart + threadIdx.x];
        // a species code out of range makes every total NaN
        if (atomicOr(&s->bad, 0u) != 0u)
            v = __longlong_as_double(0x7ff8000000000000ll);
        totals[threadIdx.x] = v;
    }
}

std::mutex g_lock;
Scratch *g_addr[kMaxDevices] = {};

// Message of the calling thread's last failed call (a fixed buffer: nothing is
// allocated to report a failure); md_last_error(NULL) returns it.
thread_local char t_msg[256] = "";

int fail(int code, const char *m)
{
    snprintf(t_msg, sizeof t_msg, "%s", m);
    return code;
}

}  // namespace

// The message of the calling thread's last md_forces_noalloc failure ("" if
// its last call succeeded); md_api.cu returns it from md_last_error(NULL).
const char *md_noalloc_message() { return t_msg; }

extern "C" int md_forces_noalloc(const md_params *p, int64_t n, double box, const int32_t *species,
                                 const double *pos, double *force, double *energy, double *totals,
                                 void *cuda_stream)
{
    t_msg[0] = '\0';
    if (!p || !species || !pos || !force || !totals)
        return fail(MD_E_INVAL, "md_forces_noalloc: null argument");
    if (!(p->precision >= MD_PREC_FP64 && p->precision <= MD_PREC_FP32))
        return fail(MD_E_INVAL, "md_forces_noalloc: unknown precision mode");
    if (n < 2)
        return fail(MD_E_INVAL, "md_forces_noalloc: need at least 2 particles");
    if (n > MD_NOALLOC_MAX_N)
        return fail(MD_E_INVAL, "md_forces_noalloc: n exceeds MD_NOALLOC_MAX_N (1048576), the size of its "
                                "fixed scratch area; use md_create / md_compute_forces instead");
    if (p->n_species < 1 || p->n_species > 2)
        return fail(MD_E_INVAL, "md_forces_noalloc: n_species must be 1 or 2");
    if (p->smooth_h != 0.0)
        return fail(MD_E_INVAL, "md_forces_noalloc: the smoothed potential (smooth_h > 0) is not supported; "
                                "use md_create / md_compute_forces");
    Pot pot;
    double rcmax = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int x = a < p->n_species ? a : p->n_species - 1, y = b < p->n_species ? b : p->n_species - 1;
            const double eps = p->eps[x][y], sig = p->sigma[x][y], rc = p->rcut[x][y];
            if (!(sig > 0.0) || !(rc > 0.0))
                return fail(MD_E_INVAL, "md_forces_noalloc: sigma and rcut must be positive");
            const double sr2 = sig * sig / (rc * rc), sr6 = sr2 * sr2 * sr2;
            const int k = a * 2 + b;
            pot.rc2[k] = rc * rc;
            pot.sig2[k] = sig * sig;
            pot.eps4[k] = 4.0 * eps;
            pot.eps48[k] = 48.0 * eps;
            pot.shift[k] = p->shift ? 4.0 * eps * (sr6 * sr6 - sr6) : 0.0;
            rcmax = rc > rcmax ? rc : rcmax;
        }
    if (!(box > 2.0 * rcmax) || !(box < 1e300))
        return fail(MD_E_INVAL, "md_forces_noalloc: box must be finite and exceed twice the largest cutoff");

    // once per device, with that device current: the scratch array's address
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(MD_E_CUDA, "md_forces_noalloc: no usable current device");
    Scratch *s;
    {
        std::lock_guard<std::mutex> lk(g_lock);
        if (!g_addr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr)
                return fail(MD_E_CUDA, "md_forces_noalloc: cudaGetSymbolAddress of the scratch area failed");
            g_addr[dev] = (Scratch *)ptr;
        }
        s = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    static_assert(offsetof(Scratch, bad) == offsetof(Scratch, ticket) + sizeof(unsigned int), "adjacent words");
    if (cudaMemsetAsync(&s->ticket, 0, 2 * sizeof(unsigned int), st) != cudaSuccess)
        return fail(MD_E_CUDA, "md_forces_noalloc: clearing the scratch ticket failed");
    const int grid = (int)((n + kBlock - 1) / kBlock);
    const int nsp = p->n_species;
    if (p->precision == MD_PREC_FP64)
        k_forces_allpairs<true><<<grid, kBlock, 0, st>>>(pot, (int)n, nsp, box, species, pos, force, energy, totals,
                                                          s);
    else
        k_forces_allpairs<false><<<grid, kBlock, 0, st>>>(pot, (int)n, nsp, box, species, pos, force, energy, totals,
                                                           s);
    if (cudaGetLastError() != cudaSuccess)
        return fail(MD_E_CUDA, "md_forces_noalloc: kernel launch failed");
    return MD_OK;
}
