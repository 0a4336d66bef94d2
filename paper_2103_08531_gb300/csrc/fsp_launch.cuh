// fsp_launch.cuh -- host helpers shared by the pass launchers (fsp_axis*.cu):
// building a launch's work list and splitting many items into launches.
#pragma once

#include "fsp_passes.cuh"

#include <algorithm>

namespace fsp {

// Work list of items[0..n): item i owns units [offs[i], offs[i+1]).
template <int MAXI>
inline Work<MAXI> make_work(const PassArgs *items, int n, int (*units)(const PassArgs &))
{
    Work<MAXI> w;
    w.nitems = n;
    w.offs[0] = 0;
    for (int i = 0; i < n; ++i) {
        w.item[i] = items[i];
        w.offs[i + 1] = w.offs[i] + units(items[i]);
    }
    return w;
}

// SM count of the current device (looked up once).
inline int sm_count()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    return sms;
}

// Runs body(work) for one item (Work<1>) or for items in chunks of BATCH_MAX
// (Work<BATCH_MAX>); stops at the first nonzero return.
template <class F>
inline int chunked(const PassArgs *items, int n, int (*units)(const PassArgs &), F body)
{
    if (n == 1) {
        Work<1> w = make_work<1>(items, 1, units);
        return body(w);
    }
    for (int i = 0; i < n; i += BATCH_MAX) {
        const int m = std::min(BATCH_MAX, n - i);
        Work<BATCH_MAX> w = make_work<BATCH_MAX>(items + i, m, units);
        int e = body(w);
        if (e) return e;
    }
    return 0;
}

} // namespace fsp
