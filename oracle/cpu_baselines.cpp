// CPU comparison sorts for the benchmark's baseline leg -- TEST AND
// MEASUREMENT INFRASTRUCTURE ONLY, never linked by the GPU library.
//
// Section 5 (Table 1) sets the GPU against a CPU quicksort; the oracle's
// median-of-three quicksort (oracle.c) plays that part on one core.  These
// are the modern references beside it:
//   cpu_std_sort_u32       std::sort on one core;
//   cpu_parallel_sort_u32  the array cut into one contiguous chunk per
//                          thread, each chunk std::sort-ed on its own
//                          std::thread, then the sorted runs merged pairwise
//                          (std::merge), the merges of one level running in
//                          parallel, ping-ponging through a scratch buffer.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

extern "C" {

void cpu_std_sort_u32(uint32_t* keys, uint64_t n) { std::sort(keys, keys + n); }

// Returns 0 on success, -1 if the scratch buffer cannot be allocated.
int cpu_parallel_sort_u32(uint32_t* keys, uint64_t n, int threads)
{
    if (threads < 1) threads = 1;
    if (n < 2) return 0;
    if ((uint64_t)threads > n / 2) threads = (int)(n / 2 > 0 ? n / 2 : 1);
    // run boundaries: threads contiguous chunks
    std::vector<uint64_t> cut(threads + 1);
    for (int t = 0; t <= threads; ++t) cut[t] = n * (uint64_t)t / (uint64_t)threads;
    {
        std::vector<std::thread> pool;
        for (int t = 0; t < threads; ++t)
            pool.emplace_back([=, &cut] { std::sort(keys + cut[t], keys + cut[t + 1]); });
        for (auto& th : pool) th.join();
    }
    std::vector<uint32_t> scratch;
    try {
        scratch.resize(n);
    } catch (...) {
        return -1;
    }
    uint32_t* src = keys;
    uint32_t* dst = scratch.data();
    while (cut.size() > 2) {
        std::vector<uint64_t> next;
        std::vector<std::thread> pool;
        for (size_t r = 0; r + 1 < cut.size(); r += 2) {
            next.push_back(cut[r]);
            if (r + 2 < cut.size()) {
                const uint64_t a = cut[r], b = cut[r + 1], c = cut[r + 2];
                pool.emplace_back([=] { std::merge(src + a, src + b, src + b, src + c, dst + a); });
            } else {  // an odd run out: carried over to the next level
                const uint64_t a = cut[r], b = cut[r + 1];
                pool.emplace_back([=] { std::memcpy(dst + a, src + a, (b - a) * sizeof(uint32_t)); });
            }
        }
        next.push_back(cut.back());
        for (auto& th : pool) th.join();
        cut.swap(next);
        std::swap(src, dst);
    }
    if (src != keys) std::memcpy(keys, src, n * sizeof(uint32_t));
    return 0;
}

}  // extern "C"
