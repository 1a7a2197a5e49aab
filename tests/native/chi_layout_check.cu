// Host-side check of the attribute packing and of chi on packed words (Eq. 4-5): for
// random layouts (a byte per attribute for m <= 4, bit fields otherwise), random object
// codes and random query codes (matching, mismatching, above the largest object code,
// and the wildcard 255), chi_packed on the packed words must equal the number of
// positions whose codes differ, open positions excluded.  Prints "ok <pairs>" or the
// first failing case.
#include <cstdio>
#include <random>

#include "nhq_internal.cuh"

using namespace nhq;

int main() {
    std::mt19937_64 rng(20260601);
    long checked = 0;
    for (int trial = 0; trial < 4000; ++trial) {
        const int m = 1 + (int)(rng() % 32);
        AttrLayout L;
        const bool bytes = m <= 4 && (rng() & 1);
        if (bytes) {
            L = byte_layout(m);
        } else {
            uint8_t maxc[kMaxAttr] = {};
            const int cap = 1 << (1 + rng() % 8);  // largest codes up to 1..255
            for (int j = 0; j < m; ++j)
                maxc[j] = (uint8_t)(rng() % (cap < 256 ? cap : 255));
            if (!compact_layout(m, maxc, &L))
                continue;  // needs more than 32 bits
        }
        nhq_weights wts{NHQ_W_CONSTANT, 1.f, 1.f};
        Fusion w = make_fusion(wts, L);
        w.wild = (int)(rng() & 1);
        Fusion wobj = w;
        wobj.wild = 0;
        for (int rep = 0; rep < 50; ++rep) {
            uint8_t a[kMaxAttr], q[kMaxAttr];
            for (int j = 0; j < m; ++j) {
                a[j] = (uint8_t)(rng() % ((unsigned)L.maxc[j] + 1u));
                switch (rng() % 4) {
                case 0: q[j] = a[j]; break;
                case 1: q[j] = (uint8_t)(rng() % ((unsigned)L.maxc[j] + 1u)); break;
                case 2: q[j] = (uint8_t)(L.maxc[j] + (rng() % (256u - L.maxc[j]))); break;
                default: q[j] = 255; break;
                }
            }
            uint32_t hi_obj, hi;
            const uint32_t wa = pack_query_word(a, wobj, &hi_obj);  // objects: no capping occurs
            const uint32_t wq = pack_query_word(q, w, &hi);
            int want = 0;
            for (int j = 0; j < m; ++j)
                if (!(w.wild && q[j] == 255))
                    want += a[j] != q[j] ? 1 : 0;
            const int got = chi_packed(wa, wq, hi, w.lo);
            if (got != want || hi_obj != L.hi) {
                std::printf("FAIL m=%d bytes=%d wild=%d chi=%d want=%d\n", m, (int)bytes, w.wild,
                            got, want);
                return 1;
            }
            ++checked;
        }
    }
    std::printf("ok %ld\n", checked);
    return 0;
}
