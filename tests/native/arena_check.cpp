// Host-pool arena checks (compiled and run by tests/test_arena.py): the
// quarantine withholds bad ranges where they are free and when their blocks
// are released, and no allocation ever overlaps a withheld range.
#include <cstdio>
#include <cstdlib>

#include "rt.hpp"

static int fails = 0;
#define EXPECT(c)                                                 \
    do {                                                          \
        if (!(c)) {                                               \
            std::printf("FAILED line %d: %s\n", __LINE__, #c);     \
            ++fails;                                              \
        }                                                         \
    } while (0)

int main() {
    const size_t MB = (size_t)1 << 20;
    Arena a;
    a.init(64 * MB, nullptr);
    a.oldest_first = true;
    size_t o1, o2, o3;
    FenceSet f;
    EXPECT(a.alloc(8 * MB, &o1, &f));
    EXPECT(a.alloc(8 * MB, &o2, &f));
    EXPECT(a.alloc(8 * MB, &o3, &f));
    // a range partly in use (o2's block) and partly free (beyond o3's block)
    a.quarantine(o2, 8 * MB);
    a.quarantine(o3 + 8 * MB, 4 * MB);
    EXPECT(a.withheld == 4 * MB);  // only the free part so far
    a.release(o2, 8 * MB, FenceSet());
    EXPECT(a.withheld == 12 * MB);  // o2's block joined when released
    // every later allocation avoids the withheld ranges
    std::vector<size_t> got;
    size_t off;
    while (a.alloc(4 * MB, &off, &f)) got.push_back(off);
    for (size_t g : got) {
        const bool in_o2 = g < o2 + 8 * MB && g + 4 * MB > o2;
        const bool in_q2 = g < o3 + 12 * MB && g + 4 * MB > o3 + 8 * MB;
        EXPECT(!in_o2 && !in_q2);
    }
    EXPECT(got.size() * 4 * MB + a.withheld + 16 * MB == 64 * MB);  // o1, o3 still held
    // releasing and re-allocating never hands out a withheld byte
    for (size_t g : got) a.release(g, 4 * MB, FenceSet());
    a.coalesce();
    size_t big;
    EXPECT(a.alloc(24 * MB, &big, &f));
    EXPECT(!(big < o2 + 8 * MB && big + 24 * MB > o2));
    // when the pool runs short, the quarantine gives its ranges back
    const size_t before = a.withheld;
    EXPECT(before > 0);
    a.release_quarantine();
    EXPECT(a.withheld == 0 && a.bad.empty());
    size_t freed = 0;
    for (auto &kv : a.free_) freed += kv.second.size;
    EXPECT(freed + a.used == a.cap);
    std::printf("%s\n", fails ? "arena checks failed" : "arena checks ok");
    return fails ? 1 : 0;
}
