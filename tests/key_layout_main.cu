// key_layout_main.cu -- host-only check of the library's grid-key layout
// (CellKeyLayout and GridMap in csrc/fec_internal.cuh), compiled with nvcc and
// run on the CPU by tests/test_key_layout.py; nothing here touches a GPU.
//
// The cell key groups the columns (c0, c1) in bricks and keeps c2 lowest.
// For random bit widths, axis orders and coordinates this checks that
//   - decode(column(c0, c1) | c2) gives back (c0, c1, c2), and the column
//     key has no bits of c2;
//   - the next cell of a column has the next key (c2 + 1 <-> key + 1);
//   - the slab of c0 (its brick row) is the key's top field;
//   - GridMap::key_of puts each original axis's coordinate where the cell
//     key expects the permuted one, with the sub-cell bits below, and
//     unpack() recovers the quantised point from key and payload, for 32-
//     and 64-bit keys;
// and, exhaustively for small widths, that the layout is a bijection that
// keeps every column's cells consecutive.
// Prints "checks=<n> failures=<m>" and exits non-zero on any failure.
#include <cstdio>
#include <cstdint>
#include <set>

#include "fec_internal.cuh"

using namespace fec;

namespace {

uint64_t g_state = 0x9E3779B97F4A7C15ull;
uint64_t next_u64()
{
    g_state ^= g_state << 13;
    g_state ^= g_state >> 7;
    g_state ^= g_state << 17;
    return g_state;
}
uint64_t below(uint64_t bound) { return bound ? next_u64() % bound : 0; }

uint64_t checks = 0, failures = 0;
void expect(bool ok, const char *what, unsigned b0, unsigned b1, unsigned b2)
{
    ++checks;
    if (!ok && failures++ < 20) std::printf("FAIL %s (bits %u %u %u)\n", what, b0, b1, b2);
}

Plan make_plan(unsigned b0, unsigned b1, unsigned b2, const int perm[3])
{
    Plan p{};
    p.bits[0] = b0;
    p.bits[1] = b1;
    p.bits[2] = b2;
    for (int i = 0; i < 3; ++i) p.perm[i] = perm[i];
    return p;
}

template <typename KeyT>
void check_grid_map(const Plan &plan, unsigned b0, unsigned b1, unsigned b2, int S)
{
    CellKeyLayout L;
    L.load(&plan);
    Params prm{};
    prm.S = S;
    prm.h = S / 2;
    Frame fr{};
    fr.lo[0] = -5000;
    fr.lo[1] = 123;
    fr.lo[2] = 77777;
    GridMap g;
    g.load(&plan, prm, fr);
    const unsigned bits[3] = {b0, b1, b2};
    for (int t = 0; t < 40; ++t) {
        uint32_t c[3], off[3];  // per original axis
        uint64_t cp[3];         // per permuted axis
        for (int p = 0; p < 3; ++p) {
            const int a = plan.perm[p];
            c[a] = (uint32_t)below(1ull << bits[p]);
            cp[p] = c[a];
        }
        for (int a = 0; a < 3; ++a) off[a] = (uint32_t)below((uint64_t)S);
        const KeyT key = g.key_of<KeyT>(c, off);
        const uint64_t ck = (uint64_t)key >> 3;
        expect(ck == (L.column(cp[0], cp[1]) | cp[2]), "key_of matches the cell key", b0, b1, b2);
        uint32_t code = 0;  // sub-cell bits: bit 2 = p0 ... bit 0 = p2
        for (int p = 0; p < 3; ++p)
            code |= (off[plan.perm[p]] >= (uint32_t)prm.h ? 1u : 0u) << (2 - p);
        expect(((uint64_t)key & 7u) == code, "sub-cell code bits", b0, b1, b2);
        const uint32_t idx = (uint32_t)below(1u << 30);
        int32_t q[3];
        g.unpack<KeyT>(key, g.payload_of(off, idx), q);
        for (int a = 0; a < 3; ++a)
            expect(q[a] == fr.lo[a] + (int32_t)(c[a] * (uint32_t)S) + (int32_t)off[a], "unpack", b0, b1,
                   b2);
    }
}

void check_layout(unsigned b0, unsigned b1, unsigned b2, const int perm[3])
{
    const Plan plan = make_plan(b0, b1, b2, perm);
    CellKeyLayout L;
    L.load(&plan);
    for (int t = 0; t < 60; ++t) {
        const uint64_t c0 = below(1ull << b0), c1 = below(1ull << b1), c2 = below(1ull << b2);
        const uint64_t col = L.column(c0, c1);
        expect((col & ((1ull << b2) - 1)) == 0, "column key has no c2 bits", b0, b1, b2);
        unsigned long long d0, d1, d2;
        L.decode(col | c2, d0, d1, d2);
        expect(d0 == c0 && d1 == c1 && d2 == c2, "decode(column | c2)", b0, b1, b2);
        expect(L.slab_of(c0) == ((col | c2) >> (b2 + b1 + L.B0)), "slab is the top field", b0, b1, b2);
        if (c2 + 1 < (1ull << b2)) {
            L.decode((col | c2) + 1, d0, d1, d2);
            expect(d0 == c0 && d1 == c1 && d2 == c2 + 1, "next cell of a column", b0, b1, b2);
        }
    }
    const int S = 1 + (int)below(1024);
    if (b0 + b1 + b2 + 3 <= 32) check_grid_map<uint32_t>(plan, b0, b1, b2, S);
    check_grid_map<unsigned long long>(plan, b0, b1, b2, S);
}

void check_bijection(unsigned b0, unsigned b1, unsigned b2)
{
    const int perm[3] = {0, 1, 2};
    const Plan plan = make_plan(b0, b1, b2, perm);
    CellKeyLayout L;
    L.load(&plan);
    std::set<uint64_t> keys;
    bool consecutive = true;
    for (uint64_t c0 = 0; c0 < (1ull << b0); ++c0)
        for (uint64_t c1 = 0; c1 < (1ull << b1); ++c1)
            for (uint64_t c2 = 0; c2 < (1ull << b2); ++c2) {
                const uint64_t k = L.column(c0, c1) | c2;
                keys.insert(k);
                consecutive = consecutive && k == L.column(c0, c1) + c2;
            }
    expect(keys.size() == (1ull << (b0 + b1 + b2)), "bijection", b0, b1, b2);
    expect(*keys.rbegin() < (1ull << (b0 + b1 + b2)), "keys within their bits", b0, b1, b2);
    expect(consecutive, "a column's cells are consecutive", b0, b1, b2);
}

}  // namespace

int main()
{
    const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int t = 0; t < 3000; ++t) {
        unsigned b[3];
        for (int i = 0; i < 3; ++i) b[i] = (t % 3 == 0) ? (unsigned)below(6) : (unsigned)below(22);
        if (b[0] + b[1] + b[2] > 58) continue;
        check_layout(b[0], b[1], b[2], perms[t % 6]);
    }
    for (unsigned b0 = 0; b0 <= 6; ++b0)
        for (unsigned b1 = 0; b1 <= 6; ++b1)
            for (unsigned b2 = 0; b2 <= 3; ++b2) check_bijection(b0, b1, b2);
    std::printf("checks=%llu failures=%llu\n", (unsigned long long)checks, (unsigned long long)failures);
    return failures ? 1 : 0;
}
