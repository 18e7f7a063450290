// Host-side checks of the chunk tables of the force and step kernels
// (paper_0912_3824_gb300/csrc/md_tables.h): the launch orders are
// permutations of the chunks, blocks that share an SM get neighbouring
// chunks, and the step kernel's sweeping table covers every chunk once with
// padding only at the end of a block's rows.  Prints "ok" or the first
// failure; exit status 0 on success.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "md_tables.h"

static int fails = 0;
#define EXPECT(c, ...)                                       \
    do {                                                     \
        if (!(c) && fails++ < 10) {                          \
            std::printf("FAIL %s:%d: ", __FILE__, __LINE__); \
            std::printf(__VA_ARGS__);                        \
            std::printf("\n");                               \
        }                                                    \
    } while (0)

static std::vector<int4> make_chunks(int nb, int per_chunk)
{
    std::vector<int4> c;
    for (int b = 0; b < nb; ++b)
        c.push_back(mdt::mk4(b * per_chunk, (b + 1) * per_chunk, 0, 0));
    return c;
}

static void check_order(int nb, int nsm, int resident)
{
    const std::vector<int4> ch = make_chunks(nb, 64);
    const std::vector<int4> o = mdt::sm_block_order(ch, nsm, resident);
    EXPECT((int)o.size() == nb, "order size %d != %d", (int)o.size(), nb);
    std::vector<int> seen(nb, 0);
    for (int p = 0; p < nb; ++p) {
        const int c = o[p].w;
        EXPECT(c >= 0 && c < nb, "chunk index %d out of range", c);
        if (c < 0 || c >= nb)
            return;
        seen[c] += 1;
        EXPECT(o[p].x == ch[c].x && o[p].y == ch[c].y, "row %d does not carry chunk %d", p, c);
    }
    for (int c = 0; c < nb; ++c)
        EXPECT(seen[c] == 1, "chunk %d appears %d times (nb %d)", c, seen[c], nb);
    if (nsm > 1 && nb > nsm && nb <= resident)       // one wave: blocks p, p + nsm, ... consecutive
        for (int p = 0; p + nsm < nb; ++p)
            EXPECT(o[p + nsm].w == o[p].w + 1, "blocks %d and %d: chunks %d, %d", p, p + nsm, o[p].w,
                   o[p + nsm].w);
}

static void check_step_table(int nb, int nsm, int per_sm)
{
    const std::vector<int4> ch = make_chunks(nb, 64);
    const std::vector<int4> order = mdt::sm_block_order(ch, nsm, nsm * per_sm);
    int nblk = 0, cpb = 0;
    const std::vector<int4> one = mdt::step_table(order, ch, false, nsm, per_sm, nblk, cpb);
    EXPECT(nblk == nb && cpb == 1 && one.size() == order.size(), "one block per chunk: %d blocks, cpb %d", nblk,
           cpb);
    const std::vector<int4> rows = mdt::step_table(order, ch, true, nsm, per_sm, nblk, cpb);
    EXPECT((int)rows.size() == nblk * cpb, "rows %d != %d x %d", (int)rows.size(), nblk, cpb);
    EXPECT((int)rows.size() < 2 * nb + 1, "rows %d exceed twice the chunks %d", (int)rows.size(), nb);
    EXPECT(nblk <= nb && nblk <= nsm * per_sm, "blocks %d (chunks %d, resident %d)", nblk, nb, nsm * per_sm);
    std::vector<int> seen(nb, 0);
    for (int b = 0; b < nblk; ++b) {
        bool pad = false;
        for (int q = 0; q < cpb; ++q) {
            const int4 r = rows[(size_t)b * cpb + q];
            if (r.w < 0) {
                pad = true;
                continue;
            }
            EXPECT(!pad, "block %d: a chunk after padding", b);
            EXPECT(r.w < nb, "chunk index %d out of range", r.w);
            if (r.w >= nb)
                continue;
            seen[r.w] += 1;
            EXPECT(r.x == ch[r.w].x && r.y == ch[r.w].y, "block %d row %d does not carry chunk %d", b, q, r.w);
        }
    }
    for (int c = 0; c < nb; ++c)
        EXPECT(seen[c] == 1, "sweep: chunk %d appears %d times (nb %d, nsm %d, per_sm %d)", c, seen[c], nb, nsm,
               per_sm);
    // the blocks of one SM group (s, s + g, s + 2 g, ... with g groups) take
    // side by side chunks of one consecutive run
    const int g = nblk < nsm ? nblk : nsm;
    const int per = nblk / g;
    for (int s = 0; s < g; ++s)
        for (int q = 0; q < cpb; ++q)
            for (int k = 0; k + 1 < per; ++k) {
                const int4 a = rows[(size_t)(s + k * g) * cpb + q], b = rows[(size_t)(s + (k + 1) * g) * cpb + q];
                if (a.w >= 0 && b.w >= 0)
                    EXPECT(b.w == a.w + 1, "group %d row %d: blocks %d, %d take chunks %d, %d", s, q, k, k + 1, a.w,
                           b.w);
            }
}

int main()
{
    const int nsm = 152;
    const int sizes[] = {1, 5, 151, 152, 153, 500, 1024, 1063, 1064, 1065, 2048, 8192, 16385};
    for (int nb : sizes)
        for (int per_sm : {1, 5, 7, 9}) {
            check_order(nb, nsm, nsm * per_sm);
            check_step_table(nb, nsm, per_sm);
        }
    unsigned int x = 12345u;
    for (int t = 0; t < 300; ++t) {
        x = x * 1664525u + 1013904223u;
        const int nb = 1 + (int)(x % 20000u);
        x = x * 1664525u + 1013904223u;
        const int ns = 1 + (int)(x % 200u);
        x = x * 1664525u + 1013904223u;
        const int ps = 1 + (int)(x % 10u);
        check_order(nb, ns, ns * ps);
        check_step_table(nb, ns, ps);
    }
    if (fails) {
        std::printf("%d failures\n", fails);
        return 1;
    }
    std::printf("ok\n");
    return 0;
}
