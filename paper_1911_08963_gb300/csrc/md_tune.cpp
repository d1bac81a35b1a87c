// md_tune.cpp -- md_batch_tune: the autotuner of md_batch's schedule.
//
// md_batch's shared schedule has three knobs whose best values depend on the batch's shapes
// and on the GPU: the combinations per work item (chunk_log2), the blocks per SM of the
// shared round kernels, and the estimated work from which a code runs on its own with the
// tensor-core levels (batch_heavy).  The tuner times md_batch itself on deterministic samples
// of the batch -- the light codes for the first two knobs, the light codes together with the
// mid-weight ones (the codes the threshold moves) for the third -- and keeps the fastest
// choice.  Choices are cached in a small JSON file, one entry per (batch shape, work budget,
// GPU), so a batch of a known shape is not timed again.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "md_internal.h"

namespace mdl {
namespace {

// Estimated work of every code (the estimator of md_batch's admission), on all host cores;
// -1 for a code that fails validation.
std::vector<double> estimates(const md_code *codes, int count) {
    std::vector<double> est(count, -1.0);
    const int nt = std::max(1, std::min<int>((int)std::thread::hardware_concurrency(), count / 16 + 1));
    std::atomic<int> next{0};
    auto work = [&]() {
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= count) break;
            Code c;
            if (build_code(codes[i].G, codes[i].n, codes[i].k, &c) == MD_OK) est[i] = estimate_work(c, nullptr, nullptr);
        }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; t++) th.emplace_back(work);
    work();
    for (auto &t : th) t.join();
    return est;
}

// Up to `want` of the codes whose estimate lies in [lo, hi), evenly spaced in batch order.
std::vector<md_code> sample(const md_code *codes, const std::vector<double> &est, double lo, double hi, int want) {
    std::vector<int> idx;
    for (int i = 0; i < (int)est.size(); i++)
        if (est[i] >= lo && est[i] < hi) idx.push_back(i);
    std::vector<md_code> out;
    if (idx.empty() || want <= 0) return out;
    const int n = std::min<int>(want, (int)idx.size());
    for (int s = 0; s < n; s++) out.push_back(codes[idx[(size_t)s * idx.size() / n]]);
    return out;
}

// Wall time of md_batch on `codes` (the fastest of `reps` runs), or a negative value on error.
double time_batch(const std::vector<md_code> &codes, const md_options &o, int reps) {
    if (codes.empty()) return 0.0;
    std::vector<int> d(codes.size()), st(codes.size());
    double best = -1.0;
    for (int r = 0; r < reps; r++) {
        const auto t0 = std::chrono::steady_clock::now();
        const int rc = md_batch(codes.data(), (int)codes.size(), &o, d.data(), nullptr, st.data());
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (rc != MD_OK) return -1.0 - rc;
        if (best < 0 || dt < best) best = dt;
    }
    return best;
}

// ---- the cache: {"key": {"chunk_log2": c, "blocks_per_sm": b, "batch_heavy": h, ...}, ...}
// Keys are plain strings (no quotes or backslashes); each value is a flat object.
std::map<std::string, std::string> read_cache(const char *path) {
    std::map<std::string, std::string> out;
    FILE *f = path ? std::fopen(path, "rb") : nullptr;
    if (!f) return out;
    std::string txt;
    char buf[4096];
    size_t nr;
    while ((nr = std::fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, nr);
    std::fclose(f);
    size_t p = txt.find('{');
    while (p != std::string::npos) {
        const size_t k0 = txt.find('"', p + 1);
        if (k0 == std::string::npos) break;
        const size_t k1 = txt.find('"', k0 + 1);
        const size_t v0 = k1 == std::string::npos ? k1 : txt.find('{', k1);
        const size_t v1 = v0 == std::string::npos ? v0 : txt.find('}', v0);
        if (v1 == std::string::npos) break;
        out[txt.substr(k0 + 1, k1 - k0 - 1)] = txt.substr(v0, v1 - v0 + 1);
        p = v1;
    }
    return out;
}

bool field(const std::string &obj, const char *name, unsigned long long *val) {
    const std::string pat = std::string("\"") + name + "\"";
    const size_t p = obj.find(pat);
    if (p == std::string::npos) return false;
    const size_t c = obj.find(':', p + pat.size());
    if (c == std::string::npos) return false;
    char *end = nullptr;
    const unsigned long long v = std::strtoull(obj.c_str() + c + 1, &end, 10);
    if (end == obj.c_str() + c + 1) return false;
    *val = v;
    return true;
}

int write_cache(const char *path, const std::map<std::string, std::string> &entries) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return MD_EINVAL;
    std::fputs("{\n", f);
    size_t i = 0;
    for (const auto &e : entries)
        std::fprintf(f, "  \"%s\": %s%s\n", e.first.c_str(), e.second.c_str(), ++i < entries.size() ? "," : "");
    std::fputs("}\n", f);
    std::fclose(f);
    return std::rename(tmp.c_str(), path) == 0 ? MD_OK : MD_EINVAL;
}

}  // namespace
}  // namespace mdl

using namespace mdl;

extern "C" int md_batch_tune_key(const md_code *codes, int count, char *key, size_t len) {
    if (!codes || count < 1 || !key || len == 0) return MD_EINVAL;
    int nlo = 1 << 30, nhi = 0, klo = 1 << 30, khi = 0;
    for (int i = 0; i < count; i++) {
        nlo = std::min(nlo, codes[i].n);
        nhi = std::max(nhi, codes[i].n);
        klo = std::min(klo, codes[i].k);
        khi = std::max(khi, codes[i].k);
    }
    int lc = 0;
    while ((1 << lc) < count) lc++;
    const int w = std::snprintf(key, len, "n%d-%d k%d-%d c2^%d", nlo / 16 * 16, (nhi + 15) / 16 * 16, klo / 8 * 8,
                                (khi + 7) / 8 * 8, lc);
    return w > 0 && (size_t)w < len ? MD_OK : MD_EINVAL;
}

extern "C" int md_batch_tune(const md_code *codes, int count, const md_options *base, const char *cache_path,
                             md_options *tuned) {
    if (!codes || count < 1 || !tuned) return MD_EINVAL;
    md_options o;
    if (base) o = *base; else md_options_init(&o);
    o.batch_mode = 0;
    char shape[128];
    int rc = md_batch_tune_key(codes, count, shape, sizeof(shape));
    if (rc != MD_OK) return rc;
    int dev = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return MD_ECUDA;
    }
    std::string key = std::string(shape) + " | budget " + std::to_string((unsigned long long)o.work_budget) + " | " +
                      prop.name;
    for (char &ch : key)
        if (ch == '"' || ch == '\\') ch = '_';
    std::map<std::string, std::string> cache = read_cache(cache_path);
    auto hit = cache.find(key);
    unsigned long long c = 0, b = 0, h = 0;
    if (hit != cache.end() && field(hit->second, "chunk_log2", &c) && field(hit->second, "blocks_per_sm", &b) &&
        field(hit->second, "batch_heavy", &h)) {
        *tuned = o;
        tuned->chunk_log2 = (int)c;
        tuned->blocks_per_sm = (int)b;
        tuned->batch_heavy = h;
        return MD_OK;
    }

    const std::vector<double> est = estimates(codes, count);
    const double budget = o.work_budget ? (double)o.work_budget : 1e300;
    // light codes: the shared schedule alone (no single-code runs)
    const std::vector<md_code> light = sample(codes, est, 0.0, std::min(budget, std::ldexp(1.0, 34)), 384);
    const int chunks[] = {16, 18, 20};
    const int blocks[] = {0, 2, 4};
    int best_c = 20, best_b = 0;
    double best_t = -1.0;
    for (int ci : chunks)
        for (int bi : blocks) {
            md_options t = o;
            t.chunk_log2 = ci;
            t.blocks_per_sm = bi;
            t.batch_heavy = ~0ull;
            if (time_batch(light, t, 1) < 0) return MD_ECUDA;              // warm-up (allocation, modules)
            const double dt = time_batch(light, t, 2);
            if (dt < 0) return (int)(-1.0 - dt);
            if (best_t < 0 || dt < best_t) { best_t = dt; best_c = ci; best_b = bi; }
        }
    // the threshold, on the light sample plus mid-weight codes (the ones it moves): taking a code
    // out of the shared rounds shortens them only as much as the rest of the mix allows
    std::vector<md_code> mid = sample(codes, est, std::ldexp(1.0, 30), std::min(budget, std::ldexp(1.0, 38)), 24);
    std::vector<md_code> mix = light;
    for (const md_code &c : mid) {
        bool dup = false;
        for (const md_code &l : light) dup |= l.G == c.G;
        if (!dup) mix.push_back(c);
    }
    const double heavies[] = {std::ldexp(1.0, 30), std::ldexp(1.0, 32), std::ldexp(1.0, 34), std::ldexp(1.0, 36),
                              std::ldexp(1.0, 38)};
    unsigned long long best_h = kBatchHeavyDefault;
    double best_m = -1.0;
    for (double hv : heavies) {
        md_options t = o;
        t.chunk_log2 = best_c;
        t.blocks_per_sm = best_b;
        t.batch_heavy = (unsigned long long)hv;
        const double dt = time_batch(mix, t, 1);
        if (dt < 0) return (int)(-1.0 - dt);
        if (best_m < 0 || dt < best_m) { best_m = dt; best_h = (unsigned long long)hv; }
    }
    *tuned = o;
    tuned->chunk_log2 = best_c;
    tuned->blocks_per_sm = best_b;
    tuned->batch_heavy = best_h;
    if (cache_path) {
        char val[512];
        std::snprintf(val, sizeof(val),
                      "{\"chunk_log2\": %d, \"blocks_per_sm\": %d, \"batch_heavy\": %llu, \"light_sample\": %zu, "
                      "\"light_seconds\": %.6f, \"mix_sample\": %zu, \"mix_seconds\": %.6f}",
                      best_c, best_b, best_h, light.size(), best_t, mix.size(), best_m);
        cache[key] = val;
        rc = write_cache(cache_path, cache);
        if (rc != MD_OK) return rc;
    }
    return MD_OK;
}
