// pip_tuning.cu -- the autotuners' cache: a JSON file that maps a tuning key
// (the kernel, the GPU's name and the shape of the configuration) to the tile
// shape the autotuner chose and its time, so that a later process on the same
// kind of GPU and the same shape of work skips the timing runs.  The paper has
// no counterpart (its NumPy program has nothing to tune).
//
// File format, one object:
//   { "<key>": {"variant": <int>, "ms": <float>}, ... }
// Keys are built here from plain tokens and never hold quotes.  The file is
// read whole and rewritten whole (to a temporary name, then renamed), under a
// process-wide lock; processes writing the same file at once may lose each
// other's new entries but never corrupt it.
#include <stdio.h>

#include <map>
#include <mutex>
#include <string>

#include "pip_internal.cuh"

namespace {

std::mutex g_tuning_mutex;
std::string g_tuning_path;

struct TuningEntry {
    int variant;
    float ms;
};

std::map<std::string, TuningEntry> read_cache(const std::string &path)
{
    std::map<std::string, TuningEntry> out;
    FILE *f = fopen(path.c_str(), "rb");
    if (f == nullptr) return out;
    std::string s;
    char buf[4096];
    size_t got;
    while ((got = fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, got);
    fclose(f);
    size_t pos = 0;
    for (;;) {
        // "<key>": {"variant": N, "ms": X}
        const size_t k0 = s.find('"', pos);
        if (k0 == std::string::npos) break;
        const size_t k1 = s.find('"', k0 + 1);
        if (k1 == std::string::npos) break;
        const std::string key = s.substr(k0 + 1, k1 - k0 - 1);
        const size_t brace = s.find('{', k1);
        const size_t close = s.find('}', k1);
        if (brace == std::string::npos || close == std::string::npos || close < brace) break;
        const std::string body = s.substr(brace, close - brace);
        const size_t v = body.find("\"variant\":"), m = body.find("\"ms\":");
        if (v != std::string::npos && m != std::string::npos) {
            TuningEntry e;
            if (sscanf(body.c_str() + v + 10, "%d", &e.variant) == 1 && sscanf(body.c_str() + m + 5, "%f", &e.ms) == 1)
                out[key] = e;
        }
        pos = close + 1;
    }
    return out;
}

bool write_cache(const std::string &path, const std::map<std::string, TuningEntry> &entries)
{
    const std::string tmp = path + ".tmp";
    FILE *f = fopen(tmp.c_str(), "wb");
    if (f == nullptr) return false;
    fputs("{\n", f);
    size_t i = 0;
    for (const auto &kv : entries) {
        fprintf(f, "  \"%s\": {\"variant\": %d, \"ms\": %.6f}%s\n", kv.first.c_str(), kv.second.variant,
                kv.second.ms, ++i < entries.size() ? "," : "");
    }
    fputs("}\n", f);
    const bool ok = fclose(f) == 0;
    return ok && rename(tmp.c_str(), path.c_str()) == 0;
}

}  // namespace

namespace pip {

std::string tuning_key(const pip_tables *t, const char *kernel, int64_t num_points, int pdtype)
{
    cudaDeviceProp prop;
    std::string gpu = cudaGetDeviceProperties(&prop, t->device) == cudaSuccess ? prop.name : "unknown";
    for (char &c : gpu)
        if (c == '"' || c == '\\') c = '_';
    char buf[256];
    snprintf(buf, sizeof buf, "%s|%s|polygons=%d|vertices=%d|points=%lld|vertex_type=%s|point_type=%s",
             kernel, gpu.c_str(), t->P, t->V, (long long)num_points, t->vdtype == PIP_I32 ? "i32" : "f32",
             pdtype == PIP_I32 ? "i32" : "f32");
    return buf;
}

bool tuning_lookup(const std::string &key, int *variant, float *ms)
{
    std::lock_guard<std::mutex> lock(g_tuning_mutex);
    if (g_tuning_path.empty()) return false;
    const auto entries = read_cache(g_tuning_path);
    const auto it = entries.find(key);
    if (it == entries.end()) return false;
    *variant = it->second.variant;
    *ms = it->second.ms;
    return true;
}

void tuning_store(const std::string &key, int variant, float ms)
{
    std::lock_guard<std::mutex> lock(g_tuning_mutex);
    if (g_tuning_path.empty()) return;
    auto entries = read_cache(g_tuning_path);
    entries[key] = TuningEntry{variant, ms};
    write_cache(g_tuning_path, entries);
}

}  // namespace pip

extern "C" pip_status pip_set_tuning_cache(const char *path)
{
    std::lock_guard<std::mutex> lock(g_tuning_mutex);
    g_tuning_path = path ? path : "";
    return PIP_OK;
}
