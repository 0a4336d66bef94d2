// fsp_autotune.cu -- picks a launch variant per (pass, padded length) by timing.
//
// Variants (bits): 4 = the cp.async column tiles of P1/P2/P4/P5 instead of
// the TMA-staged ones (lengths <= 512; single solves: batches keep the
// defaults); 1 = with bit 4, 8 values per thread in those tiles instead of 16
// (not 192); 2 = one CTA per SM in the persistent launches instead of as many
// as fit; 8 = without bit 4, the second radix split of the length (Plan16B:
// 8 x 16 at 128, 8 x 8 x 4 at 256, 8 x 8 x 8 at 512, instead of 16 x 8,
// 16 x 16 and 16 x 16 x 2) in the TMA tiles and the single-solve middle pass,
// and at 2n = 1024 the middle pass as two 512-point halves (p3_fwd_2h).  For the middle pass at 2n = 1024 and 2048, bit 4 selects the
// block-synchronous line kernel instead of the multi-warp-per-line one, and at
// 2n = 8192 instead of the four-step (16 x 512) pass; for P5 at 2n = 8192 it
// selects the staged block-synchronous columns instead of the four-step
// through global memory.  The table is process-wide,
// keyed by pass kind and padded length, and is read by every solve.  A small
// JSON file caches it per GPU architecture, e.g.
//   {"sm_103": {"p3_fwd/512": 0, "p4_fwd/512": 2}}
#include "fsp_internal.h"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace fsp {
int run_forward(const Plan &p, void *ws, const float *rho, float *phi, float *E, cudaStream_t st);
}

using namespace fsp;

namespace {

const int kLengths[] = {32, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096, 6144, 8192};
constexpr int kNL = sizeof(kLengths) / sizeof(kLengths[0]);
const char *kKindName[PASS_KINDS] = {"p1_fwd", "p1_adj", "p2_fwd", "p2_adj", "p3_fwd", "p3_adj", "p4_fwd", "p5_fwd"};

int g_var[PASS_KINDS][kNL] = {};
std::mutex g_mu;

int length_index(int N)
{
    for (int i = 0; i < kNL; ++i)
        if (kLengths[i] == N) return i;
    return -1;
}

std::vector<int> candidates(int kind, int N)
{
    const bool tile = kind == PASS_P1F || kind == PASS_P2F || kind == PASS_P4F || kind == PASS_P5F;
    if (N > 512) {
        if (kind == PASS_P3F && N == 1024) return {0, 2, 4, 6, 8, 10};   // 8: two 512-point halves
        if (kind == PASS_P3F && (N == 768 || N == 1536 || N == 2048)) return {0, 2, 4, 6};
        if ((kind == PASS_P3F || kind == PASS_P5F) && N == 8192) return {0, 4};
        return {0};
    }
    std::vector<int> c;
    if (tile) c = N == 192 ? std::vector<int>{0, 2, 4, 6} : std::vector<int>{0, 2, 4, 5, 6, 7};
    else if (kind == PASS_P3F || kind == PASS_P3A) c = {0, 2};
    else c = {0};
    // the second radix split (the TMA tiles and the single-solve middle pass)
    if ((tile || kind == PASS_P3F) && has_radix_plan_b(N)) c.insert(c.end(), {8, 10});
    return c;
}

std::string arch_key()
{
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "sm_unknown";
    return "sm_" + std::to_string(prop.major * 10 + prop.minor);
}

// Minimal reader for the cache format written below: "name/N": value pairs
// inside the object of the current architecture.
void load_cache(const char *path, const std::string &arch)
{
    FILE *f = path ? std::fopen(path, "r") : nullptr;
    if (!f) return;
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
    std::fclose(f);
    size_t at = text.find("\"" + arch + "\"");
    if (at == std::string::npos) return;
    size_t open = text.find('{', at), close = text.find('}', at);
    if (open == std::string::npos || close == std::string::npos || close < open) return;
    std::string body = text.substr(open + 1, close - open - 1);
    size_t pos = 0;
    while ((pos = body.find('"', pos)) != std::string::npos) {
        size_t end = body.find('"', pos + 1);
        if (end == std::string::npos) break;
        std::string key = body.substr(pos + 1, end - pos - 1);
        size_t colon = body.find(':', end);
        if (colon == std::string::npos) break;
        int val = std::atoi(body.c_str() + colon + 1);
        size_t slash = key.find('/');
        if (slash != std::string::npos) {
            std::string name = key.substr(0, slash);
            int N = std::atoi(key.c_str() + slash + 1);
            int li = length_index(N);
            for (int k = 0; k < PASS_KINDS && li >= 0; ++k)
                if (name == kKindName[k] && val >= 0 && val < 16) g_var[k][li] = val;
        }
        pos = colon + 1;
    }
}

void save_cache(const char *path, const std::string &arch, const std::map<std::string, int> &entries)
{
    if (!path) return;
    std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "{\"%s\": {", arch.c_str());
    bool first = true;
    for (const auto &kv : entries) {
        std::fprintf(f, "%s\"%s\": %d", first ? "" : ", ", kv.first.c_str(), kv.second);
        first = false;
    }
    std::fprintf(f, "}}\n");
    std::fclose(f);
    std::rename(tmp.c_str(), path);
}

} // namespace

namespace fsp {
int tuned_variant(int kind, int N)
{
    const int li = length_index(N);
    if (kind < 0 || kind >= PASS_KINDS || li < 0) return 0;
    return g_var[kind][li];
}
} // namespace fsp

// Tune the forward passes this plan uses.  mode 0: read the cache only;
// 1: read it and time the passes it lacks; 2: time every pass of the plan.
// The timing solves run on a private stream with scratch buffers allocated
// here (this call allocates; solves never do).
static int autotune(fsp_plan *plan, const char *cache_path, int mode);

extern "C" int fsp_autotune(fsp_plan *plan, const char *cache_path, int mode)
{
    return record_error(autotune(plan, cache_path, mode));
}

static int autotune(fsp_plan *plan, const char *cache_path, int mode)
{
    if (!plan || mode < 0 || mode > 2) return FSP_ERR_INVALID;
    const Plan &p = plan->p;
    const std::string arch = arch_key();
    std::lock_guard<std::mutex> lk(g_mu);
    int have_cache[PASS_KINDS][kNL] = {};
    {
        int before[PASS_KINDS][kNL];
        std::memcpy(before, g_var, sizeof(g_var));
        for (int k = 0; k < PASS_KINDS; ++k)
            for (int i = 0; i < kNL; ++i) g_var[k][i] = -1;
        load_cache(cache_path, arch);
        for (int k = 0; k < PASS_KINDS; ++k)
            for (int i = 0; i < kNL; ++i) {
                have_cache[k][i] = g_var[k][i] >= 0;
                if (!have_cache[k][i]) g_var[k][i] = before[k][i];
            }
    }
    if (mode == 0 || p.direct) return FSP_OK;

    struct Job {
        int kind, N, slot;   // slot: index of the pass in the forward pipeline (event interval)
    };
    std::vector<Job> jobs;
    if (p.three_d) {
        jobs = {{PASS_P1F, 2 * p.n0, 0}, {PASS_P2F, 2 * p.n1, 1}, {PASS_P3F, 2 * p.n2, 2},
                {PASS_P4F, 2 * p.n1, 3}, {PASS_P5F, 2 * p.n0, 4}};
    } else {
        jobs = {{PASS_P1F, 2 * p.n0, 0}, {PASS_P3F, 2 * p.n2, 1}, {PASS_P5F, 2 * p.n0, 2}};
    }
    const size_t cells = (size_t)p.n0 * p.n1 * p.n2;
    const size_t ws_bytes = fsp_plan_workspace_bytes(plan, 1, 1);
    float *rho = nullptr, *phi = nullptr, *E = nullptr;
    void *ws = nullptr;
    cudaStream_t st = nullptr;
    const int nev = (p.three_d ? 5 : 3) + 1;
    cudaEvent_t ev[8] = {};
    int rc = FSP_OK;
    if (cudaMalloc(&rho, cells * sizeof(float)) != cudaSuccess || cudaMalloc(&phi, cells * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&E, 3 * cells * sizeof(float)) != cudaSuccess || cudaMalloc(&ws, ws_bytes) != cudaSuccess)
        rc = FSP_ERR_NOMEM;
    if (rc == FSP_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = FSP_ERR_CUDA;
    for (int i = 0; i < nev && rc == FSP_OK; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) rc = FSP_ERR_CUDA;
    if (rc == FSP_OK && cudaMemsetAsync(rho, 0, cells * sizeof(float), st) != cudaSuccess) rc = FSP_ERR_CUDA;

    // private copy of the plan with events attached (the caller's plan is untouched)
    Plan q = p;
    q.n_pass_ev = nev;
    for (int i = 0; i < nev; ++i) q.pass_ev[i] = ev[i];
    auto time_pass = [&](int slot) -> float {
        for (int w = 0; w < 2; ++w) run_forward(q, ws, rho, phi, E, st);
        std::vector<float> t;
        for (int r = 0; r < 5; ++r) {
            run_forward(q, ws, rho, phi, E, st);
            cudaStreamSynchronize(st);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[slot], ev[slot + 1]);
            t.push_back(ms);
        }
        std::sort(t.begin(), t.end());
        return t[t.size() / 2];
    };
    // FSP_TUNE_LOG set: every timed variant is reported on stderr
    const bool log = std::getenv("FSP_TUNE_LOG") != nullptr;
    for (const Job &j : jobs) {
        if (rc != FSP_OK) break;
        const int li = length_index(j.N);
        if (li < 0) continue;
        if (mode == 1 && have_cache[j.kind][li]) continue;
        float best = 1e30f;
        int best_v = 0;
        for (int v : candidates(j.kind, j.N)) {
            g_var[j.kind][li] = v;
            const float ms = time_pass(j.slot);
            if (cudaGetLastError() != cudaSuccess) {
                rc = FSP_ERR_CUDA;
                break;
            }
            if (log) std::fprintf(stderr, "fsp_autotune %s/%d variant %d: %.4f ms\n", kKindName[j.kind], j.N, v, ms);
            if (ms < best) {
                best = ms;
                best_v = v;
            }
        }
        g_var[j.kind][li] = best_v;
        have_cache[j.kind][li] = 1;
    }
    if (rc == FSP_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = FSP_ERR_CUDA;
    for (int i = 0; i < nev; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    if (st) cudaStreamDestroy(st);
    cudaFree(rho);
    cudaFree(phi);
    cudaFree(E);
    cudaFree(ws);
    if (rc == FSP_OK) {
        std::map<std::string, int> entries;
        for (int k = 0; k < PASS_KINDS; ++k)
            for (int i = 0; i < kNL; ++i)
                if (have_cache[k][i]) entries[std::string(kKindName[k]) + "/" + std::to_string(kLengths[i])] = g_var[k][i];
        save_cache(cache_path, arch, entries);
    }
    return rc;
}

// Current table entry (for tests and reports): variant of pass `kind` at length N.
extern "C" int fsp_tuned_variant(int kind, int N) { return tuned_variant(kind, N); }
