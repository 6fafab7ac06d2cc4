// Autotuner of the sweep's launch shape (threads per replica, warps per CTA).
//
// Only speed depends on the shape: every shape a run accepts gives the same
// spins, energies, histograms and rows (the random numbers are keyed on the
// replica slot and the site, never on the thread that updates it). The tuner
// times each candidate shape on a short probe run of the configuration's
// lattice, format and population size, keeps the fastest, and remembers the
// choice per (L, spin format, lattice dimension, Potts q, floor(log2 R),
// batched or alone, GPU name, SM count) in this process and, if asked, in a
// text file that later processes read back.
//
// File format: one choice per line,
//   v1|L|format|dim|potts_q|r_log2|batched|sms|gpu name|group_threads|block_warps|attempts_per_ns
// later lines replace earlier ones with the same key; malformed lines are
// ignored. The file is rewritten through a temporary file and a rename.
//
// This file must be compiled with -ffp-contract=off like the engine (it
// formats and parses doubles only).
#include "../../include/pa.h"
#include "pa_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#define PA_TRY_TUNE(x)               \
    do {                             \
        pa_status s_ = (x);          \
        if (s_ != PA_OK) return s_;  \
    } while (0)

namespace {

std::mutex g_mu;
std::map<std::string, pa_tune_choice> g_mem;  // key string -> choice (this process)

std::string key_string(const pa_tune_key& k)
{
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%d|%d|%d|%d|%d|%d|%d|%.63s", k.L, k.spin_format, k.dim, k.potts_q, k.r_log2,
                  k.batched, k.sms, k.gpu);
    return std::string(buf);
}

int ilog2(long long v)
{
    int r = 0;
    while (v > 1) {
        v >>= 1;
        r++;
    }
    return r;
}

// device name and SM count of the current device, looked up once per device
bool device_of(int* sms, char name[64])
{
    static std::mutex mu;
    static std::map<int, std::pair<int, std::string>> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(dev);
    if (it == cache.end()) {
        cudaDeviceProp p;
        if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        it = cache.emplace(dev, std::make_pair(p.multiProcessorCount, std::string(p.name))).first;
    }
    *sms = it->second.first;
    std::snprintf(name, 64, "%s", it->second.second.c_str());
    return true;
}

// one line of the cache file -> (key string, choice); false if malformed
bool parse_line(const char* line, std::string* key, pa_tune_choice* c)
{
    // split on '|' into 12 fields
    std::vector<std::string> f;
    std::string cur;
    for (const char* p = line; *p && *p != '\n' && *p != '\r'; p++) {
        if (*p == '|') {
            f.push_back(cur);
            cur.clear();
        } else {
            cur.push_back(*p);
        }
    }
    f.push_back(cur);
    if (f.size() != 12 || f[0] != "v1" || f[8].empty() || f[8].size() > 63) return false;
    pa_tune_key k{};
    int* ints[7] = {&k.L, &k.spin_format, &k.dim, &k.potts_q, &k.r_log2, &k.batched, &k.sms};
    for (int i = 0; i < 7; i++) {
        char* end = nullptr;
        const long v = std::strtol(f[(size_t)i + 1].c_str(), &end, 10);
        if (!end || *end || f[(size_t)i + 1].empty()) return false;
        *ints[i] = (int)v;
    }
    std::snprintf(k.gpu, sizeof(k.gpu), "%s", f[8].c_str());
    char *e1 = nullptr, *e2 = nullptr, *e3 = nullptr;
    const long g = std::strtol(f[9].c_str(), &e1, 10), bw = std::strtol(f[10].c_str(), &e2, 10);
    const double apn = std::strtod(f[11].c_str(), &e3);
    if (!e1 || *e1 || !e2 || *e2 || !e3 || *e3 || f[9].empty() || f[10].empty() || f[11].empty()) return false;
    if (g < 1 || g > 256 || bw < 0 || bw > 8) return false;
    *key = key_string(k);
    *c = pa_tune_choice{};
    c->group_threads = (int32_t)g;
    c->block_warps = (int32_t)bw;
    c->attempts_per_ns = apn;
    c->candidates = 0;
    return true;
}

bool lookup_file(const char* path, const std::string& key, pa_tune_choice* out)
{
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        std::string k;
        pa_tune_choice c;
        if (parse_line(line, &k, &c) && k == key) {
            *out = c;  // the last matching line wins
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

pa_status store_file(const char* path, const pa_tune_key& key, const pa_tune_choice& c)
{
    const std::string ks = key_string(key);
    std::vector<std::string> keep;
    if (FILE* f = std::fopen(path, "r")) {
        char line[512];
        while (std::fgets(line, sizeof(line), f)) {
            std::string k;
            pa_tune_choice old;
            if (parse_line(line, &k, &old) && k != ks) keep.emplace_back(line);
        }
        std::fclose(f);
    }
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return PA_EINVAL;
    for (const std::string& ln : keep) std::fputs(ln.c_str(), f);
    std::fprintf(f, "v1|%d|%d|%d|%d|%d|%d|%d|%.63s|%d|%d|%.17g\n", key.L, key.spin_format, key.dim, key.potts_q,
                 key.r_log2, key.batched, key.sms, key.gpu, c.group_threads, c.block_warps, c.attempts_per_ns);
    const bool ok = std::fclose(f) == 0;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return PA_EINVAL;
    }
    return PA_OK;
}

bool gpu_name_ok(const char* s)
{
    const size_t n = strnlen(s, 64);
    if (n == 0 || n == 64) return false;
    for (size_t i = 0; i < n; i++)
        if (s[i] == '|' || s[i] == '\n' || s[i] == '\r') return false;
    return true;
}

const char* cache_path_of(const char* path)
{
    if (path && *path) return path;
    const char* env = std::getenv("PA_TUNE_CACHE");
    return (env && *env) ? env : nullptr;
}

// Sweep rate of one launch shape on a two-step probe of cfg's lattice,
// format and population (attempts per ns of the sweep kernel alone).
pa_status probe(const pa_config& cfg, int G, int bw, void* stream, double* apn)
{
    pa_config pc = cfg;
    pc.group_threads = G;
    pc.block_warps = bw;
    pc.use_graph = 0;
    pc.profile = 1;
    pc.record_histograms = 0;
    pc.capacity = 0;
    pc.theta = std::min(cfg.theta, 10);
    pc.dbeta = 0.05;
    pc.beta_f = 0.1;  // two steps
    pa_ctx* t = nullptr;
    pa_status st = pa_create(&pc, stream, &t);
    if (st != PA_OK) return st;
    st = pa_run(t);
    double ms[7];
    int64_t n[7];
    if (st == PA_OK) st = pa_phase_times(t, ms, n);
    std::vector<pa_obs> rows(4);
    int64_t nr = 0;
    if (st == PA_OK) st = pa_observables(t, rows.data(), (int64_t)rows.size(), &nr);
    pa_destroy(t);
    if (st != PA_OK) return st;
    double sites = (double)cfg.L * cfg.L * (cfg.dim == 3 ? cfg.L : 1);
    double att = 0.0;
    for (int64_t i = 1; i < nr; i++) att += sites * pc.theta * (double)rows[(size_t)i].R;
    *apn = ms[4] > 0.0 ? att / (ms[4] * 1e6) : 0.0;
    return PA_OK;
}

// candidate shapes: every threads-per-replica a format may accept (the probe
// rejects the ones this run does not), each with 2, 4 and 8 warps per CTA;
// a CTA-wide group has one shape
std::vector<std::pair<int, int>> candidates(const pa_config& cfg, bool batched)
{
    std::vector<std::pair<int, int>> out;
    if (cfg.spin_format == PA_SPIN_MSC32 || cfg.spin_format == PA_SPIN_REPLICA8) {
        out.emplace_back(1, 0);  // one shape: 32-replica groups per CTA / one thread per replica
        return out;
    }
    for (int g : {1, 2, 4, 8, 16, 32}) {
        if (batched) {
            if (pa::batch_supports(cfg.L, g)) out.emplace_back(g, 0);  // the batched sweep has 8-warp CTAs
            continue;
        }
        for (int bw : {2, 4, 8}) out.emplace_back(g, bw);
    }
    if (!batched || pa::batch_supports(cfg.L, 256)) out.emplace_back(256, 0);
    return out;
}

}  // namespace

namespace pa {

// The shape pa_autotune chose in this process for runs like cfg, if any
// (used by pa_create when the config leaves the shape open).
bool tuned_shape(const pa_config& cfg, int batched, int* G, int* bw)
{
    pa_tune_key k;
    if (pa_tune_key_of(&cfg, batched, &k) != PA_OK) return false;
    std::lock_guard<std::mutex> g(g_mu);
    auto it = g_mem.find(key_string(k));
    if (it == g_mem.end()) return false;
    *G = it->second.group_threads;
    *bw = it->second.block_warps;
    return true;
}

pa_status autotune_impl(const pa_config* cfg, int batched, const char* cache_path, void* stream, pa_tune_choice* out)
{
    if (!cfg || !out) return PA_EINVAL;
    pa_tune_key key;
    PA_TRY_TUNE(pa_tune_key_of(cfg, batched, &key));
    const std::string ks = key_string(key);
    {
        std::lock_guard<std::mutex> g(g_mu);
        auto it = g_mem.find(ks);
        if (it != g_mem.end()) {
            *out = it->second;
            out->candidates = 0;
            return PA_OK;
        }
    }
    const char* path = cache_path_of(cache_path);
    pa_tune_choice c{};
    if (path && lookup_file(path, ks, &c)) {
        std::lock_guard<std::mutex> g(g_mu);
        g_mem[ks] = c;
        *out = c;
        return PA_OK;
    }
    int best_g = 0, best_bw = 0, tried = 0;
    double best = -1.0;
    for (const auto& cand : candidates(*cfg, batched != 0)) {
        double apn = 0.0;
        const pa_status st = probe(*cfg, cand.first, cand.second, stream, &apn);
        if (st == PA_EINVAL) continue;  // a shape this run does not accept
        if (st != PA_OK) return st;
        tried++;
        if (apn > best) {
            best = apn;
            best_g = cand.first;
            best_bw = cand.second;
        }
    }
    if (tried == 0) return PA_EINVAL;
    c.group_threads = best_g;
    c.block_warps = best_bw;
    c.attempts_per_ns = best;
    c.candidates = tried;
    {
        std::lock_guard<std::mutex> g(g_mu);
        g_mem[ks] = c;
    }
    if (path) {
        const pa_status fs = store_file(path, key, c);
        if (fs != PA_OK) return fs;
    }
    *out = c;
    return PA_OK;
}

}  // namespace pa

extern "C" {

pa_status pa_tune_key_of(const pa_config* cfg, int32_t batched, pa_tune_key* out)
{
    if (!cfg || !out || cfg->R < 1) return PA_EINVAL;
    std::memset(out, 0, sizeof(*out));
    out->L = cfg->L;
    out->spin_format = cfg->spin_format;
    out->dim = cfg->dim == 3 ? 3 : 2;
    out->potts_q = cfg->potts_q;
    out->r_log2 = ilog2(cfg->R);
    out->batched = batched ? 1 : 0;
    if (!device_of(&out->sms, out->gpu)) return PA_ECUDA;
    return PA_OK;
}

pa_status pa_tune_cache_store(const char* path, const pa_tune_key* key, const pa_tune_choice* choice)
{
    if (!path || !*path || !key || !choice || !gpu_name_ok(key->gpu) || choice->group_threads < 1 ||
        choice->group_threads > 256 || choice->block_warps < 0 || choice->block_warps > 8)
        return PA_EINVAL;
    return store_file(path, *key, *choice);
}

pa_status pa_tune_cache_lookup(const char* path, const pa_tune_key* key, pa_tune_choice* out, int32_t* found)
{
    if (!path || !*path || !key || !out || !found || !gpu_name_ok(key->gpu)) return PA_EINVAL;
    pa_tune_choice c{};
    *found = lookup_file(path, key_string(*key), &c) ? 1 : 0;
    if (*found) *out = c;
    return PA_OK;
}

pa_status pa_autotune(const pa_config* cfg, const char* cache_path, void* stream, pa_tune_choice* out)
{
    return pa::autotune_impl(cfg, 0, cache_path, stream, out);
}

}  // extern "C"
