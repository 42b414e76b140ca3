// Host-side ordering of a batch's pairs (host code only).
#pragma once

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

namespace nw {

// Indices 0..n-1 ordered by ascending key, equal keys in index order: an LSD
// radix sort, 16 bits a pass, skipping the passes whose digit every key
// shares.  Linear in n; a comparison sort of the 20,000 pairs of a batch
// took milliseconds of host time on the step's path.
inline std::vector<uint32_t> radix_order(const std::vector<uint64_t> &key) {
    const size_t n = key.size();
    std::vector<uint32_t> a(n), b(n);
    for (size_t i = 0; i < n; ++i) a[i] = (uint32_t)i;
    uint64_t differ = 0;
    for (size_t i = 1; i < n; ++i) differ |= key[i] ^ key[0];
    std::vector<uint32_t> cnt(1u << 16);
    for (int sh = 0; sh < 64; sh += 16) {
        if (((differ >> sh) & 0xFFFFu) == 0) continue;
        std::fill(cnt.begin(), cnt.end(), 0u);
        for (size_t i = 0; i < n; ++i) ++cnt[(key[a[i]] >> sh) & 0xFFFFu];
        uint32_t s = 0;
        for (uint32_t &c : cnt) {
            const uint32_t t = c;
            c = s;
            s += t;
        }
        for (size_t i = 0; i < n; ++i) b[cnt[(key[a[i]] >> sh) & 0xFFFFu]++] = a[i];
        a.swap(b);
    }
    return a;
}

// The same by descending key (equal keys still in index order).
inline std::vector<uint32_t> radix_order_desc(std::vector<uint64_t> key) {
    for (uint64_t &k : key) k = ~k;
    return radix_order(key);
}

// A key that orders non-negative doubles as the values do (their bits).
inline uint64_t order_key(double x) {
    uint64_t k;
    std::memcpy(&k, &x, sizeof k);
    return x > 0.0 ? k : 0u;
}

}  // namespace nw
