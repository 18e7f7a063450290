// md_tables.h -- host-side chunk tables of the force and step kernels.
//
// Plain C++ over CUDA's int4 (x = first particle, y = end, z = replica,
// w = chunk index): no device code, so the tables can be checked on the CPU
// (tests/tables_unit.cpp).
#ifndef MD_GB300_TABLES_H
#define MD_GB300_TABLES_H

#include <vector_types.h>

#include <cstdint>
#include <vector>

namespace mdt {

inline int4 mk4(int x, int y, int z, int w)
{
    int4 v;
    v.x = x;
    v.y = y;
    v.z = z;
    v.w = w;
    return v;
}

// Launch order of the force-kernel chunks.  A launch that fits in one wave
// (at most `resident` blocks) hands its blocks to the SMs in turns: the first
// nsm blocks go one to each SM (in an order of the GPU's own, not p -> SM p),
// and the next nsm in the same order, so blocks p, p + nsm, p + 2 nsm, ...
// share an SM (per-block SM ids read on GB300); giving them consecutive chunks
// (neighbouring cells along the cell curve) lets one SM's blocks share the
// neighbour positions they gather in its L1.  A longer launch keeps the chunk
// order, so that the blocks resident at any time cover one compact region.
// Block p carries its chunk index in w, where its partial sums go, so the
// per-replica sums keep their order.
inline std::vector<int4> sm_block_order(const std::vector<int4> &chunks, int nsm, int resident)
{
    const int nb = (int)chunks.size();
    std::vector<int4> out(chunks);
    for (int c = 0; c < nb; ++c)
        out[c].w = c;
    if (nsm <= 1 || nb <= nsm || nb > resident)
        return out;
    int c = 0;
    for (int s = 0; s < nsm; ++s)
        for (int p = s; p < nb; p += nsm, ++c) {
            out[p] = chunks[c];
            out[p].w = c;
        }
    return out;
}

// Rows of the step kernel's table (see KArgs::blk_s).  With one block per
// chunk they are the force kernel's rows.  The sweeping form launches only the
// resident blocks (nsm * per_sm) and gives each group of blocks that share an
// SM (blocks s, s + nsm, s + 2 nsm, ...) one run of consecutive chunks along
// the cell curve: the per_sm blocks of group s take neighbouring chunks of its
// run side by side (block s + k nsm: chunks base_s + k, base_s + k + per_sm,
// ...), so that at any time they work on one compact region and share the
// neighbour positions they gather in the SM's L1
// (with one block per chunk, a launch longer than one wave hands each freed
// slot the next chunk, so an SM's blocks lie anywhere in the resident region).
// Each row carries its chunk index in w; a block's rows end in padding
// (w = -1).  Returns the rows, cpb per block.
inline std::vector<int4> step_table(const std::vector<int4> &order, const std::vector<int4> &chunks, bool sweep,
                                    int nsm, int per_sm, int &nblk_s, int &cpb)
{
    const int nb = (int)chunks.size();
    if (!sweep || nsm < 1 || per_sm < 1) {
        nblk_s = nb;
        cpb = 1;
        return order;
    }
    if ((int64_t)nsm * per_sm > nb) {           // fewer chunks than resident blocks: at most nb blocks
        if (nb < nsm) {
            nsm = nb;
            per_sm = 1;
        } else {
            per_sm = nb / nsm;
        }
    }
    const int resident = nsm * per_sm;           // <= nb, so the rows (< nb + resident) fit 2 nb
    nblk_s = resident;
    cpb = (nb + resident - 1) / resident;
    std::vector<int4> rows((size_t)resident * cpb, mk4(0, 0, 0, -1));
    int base = 0;
    for (int s = 0; s < nsm; ++s) {
        const int ns = nb / nsm + (s < nb % nsm ? 1 : 0);   // chunks of SM s
        for (int k = 0; k < per_sm; ++k) {
            const int b = s + k * nsm;
            for (int q = 0; q < cpb; ++q) {
                const int c = q * per_sm + k;
                if (c >= ns)
                    break;
                rows[(size_t)b * cpb + q] = chunks[base + c];
                rows[(size_t)b * cpb + q].w = base + c;
            }
        }
        base += ns;
    }
    return rows;
}

}  // namespace mdt

#endif  // MD_GB300_TABLES_H
