// Tuning cache of the batched launches (not in the paper): the launch choice
// the batch tuner measured for a class of batches, kept in a small JSON file
// so that a later process reuses it without timing again.
//
// A class is keyed by what the choice depends on: precision, standardisation,
// the GPU's SM count, and the power-of-two buckets of the largest p, the mean
// n and the number of fits.  Every entry records the library and tuning-schema
// version it was measured with; an entry of another version is not used (a
// change of the kernels invalidates the cache).  The file is read whole and
// rewritten through a temporary file and a rename, so a reader never sees a
// half-written file.  The format is fixed and written only here:
//   {"spmesl_tune_cache": 1, "entries": {
//     "<key>": {"version": "<v>", "warps_per_block": 8, "handover": 32,
//               "heavy_min_p": 4096, "heavy_heat": 32, "ms": 3.72}, ...}}
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <string>

#include "common.cuh"

namespace spmesl {
namespace {

constexpr int kTuneSchema = 1;

std::string version_tag() {
    char buf[64];
    snprintf(buf, sizeof(buf), "%d/%d", spmesl_version(), kTuneSchema);
    return buf;
}

int log2_bucket(double x) {
    if (!(x > 1.0)) return 0;
    return (int)ceil(log2(x));
}

// Text of the file, or empty.
std::string read_file(const char* path) {
    std::string s;
    FILE* f = fopen(path, "rb");
    if (!f) return s;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, n);
    fclose(f);
    return s;
}

// The number after "\"name\":" inside [from, to), or false.
bool field(const std::string& s, size_t from, size_t to, const char* name, double* out) {
    const std::string pat = std::string("\"") + name + "\":";
    const size_t at = s.find(pat, from);
    if (at == std::string::npos || at >= to) return false;
    const char* p = s.c_str() + at + pat.size();
    char* end = nullptr;
    const double v = strtod(p, &end);
    if (end == p) return false;
    *out = v;
    return true;
}

// The string after "\"name\":\"" inside [from, to), or empty.
std::string sfield(const std::string& s, size_t from, size_t to, const char* name) {
    const std::string pat = std::string("\"") + name + "\":\"";
    const size_t at = s.find(pat, from);
    if (at == std::string::npos || at >= to) return std::string();
    const size_t b = at + pat.size();
    const size_t e = s.find('"', b);
    if (e == std::string::npos || e > to) return std::string();
    return s.substr(b, e - b);
}

struct Entry {
    std::string version;
    spmesl_tune_choice c;
};

// Every well-formed entry of the file (a malformed file gives none).
std::map<std::string, Entry> parse(const std::string& s) {
    std::map<std::string, Entry> m;
    if (s.find("\"spmesl_tune_cache\":1") == std::string::npos) return m;
    size_t pos = s.find("\"entries\":{");
    if (pos == std::string::npos) return m;
    pos += 11;
    for (;;) {
        const size_t kq = s.find('"', pos);
        if (kq == std::string::npos) break;
        const size_t ke = s.find('"', kq + 1);
        if (ke == std::string::npos) break;
        const size_t ob = s.find('{', ke);
        const size_t cb = s.find('}', ke);
        if (ob == std::string::npos || cb == std::string::npos || ob > cb) break;
        Entry e{};
        e.version = sfield(s, ob, cb, "version");
        double w = 0, h = 0, mp = 0, hh = 0, ms = 0;
        if (!e.version.empty() && field(s, ob, cb, "warps_per_block", &w) &&
            field(s, ob, cb, "handover", &h) && field(s, ob, cb, "heavy_min_p", &mp) &&
            field(s, ob, cb, "heavy_heat", &hh) && field(s, ob, cb, "ms", &ms)) {
            e.c.warps_per_block = (int32_t)w;
            e.c.handover = (int32_t)h;
            e.c.heavy_min_p = (int32_t)mp;
            e.c.heavy_heat = (int32_t)hh;
            e.c.ms = (float)ms;
            e.c.from_cache = 1;
            m[s.substr(kq + 1, ke - kq - 1)] = e;
        }
        pos = cb + 1;
    }
    return m;
}

}  // namespace
}  // namespace spmesl

using namespace spmesl;

extern "C" {

int spmesl_tune_key(int precision, int standardize, int sms, int count, int max_p, double mean_n,
                    char* key, size_t len) {
    if (!key || len == 0 || count < 1 || max_p < 1 || sms < 1) return -1;
    const int n = snprintf(key, len, "prec=%d|std=%d|sms=%d|pmax=2^%d|nmean=2^%d|fits=2^%d",
                           precision, standardize ? 1 : 0, sms, log2_bucket(max_p),
                           log2_bucket(mean_n), log2_bucket(count));
    return (n < 0 || (size_t)n >= len) ? -1 : n;
}

spmesl_status spmesl_tune_cache_lookup(const char* path, const char* key, spmesl_tune_choice* out) {
    if (!path || !key || !out) return SPMESL_EINVAL;
    const std::map<std::string, Entry> m = parse(read_file(path));
    const auto it = m.find(key);
    if (it == m.end() || it->second.version != version_tag()) return SPMESL_ENOTFOUND;
    *out = it->second.c;
    return SPMESL_OK;
}

spmesl_status spmesl_tune_cache_store(const char* path, const char* key,
                                      const spmesl_tune_choice* c) {
    if (!path || !key || !c || strchr(key, '"') || strchr(key, '\\')) return SPMESL_EINVAL;
    std::map<std::string, Entry> m = parse(read_file(path));
    Entry e{};
    e.version = version_tag();
    e.c = *c;
    m[key] = e;
    std::string out = "{\"spmesl_tune_cache\":1,\"entries\":{";
    bool first = true;
    for (const auto& kv : m) {
        char buf[512];
        snprintf(buf, sizeof(buf),
                 "%s\n\"%s\":{\"version\":\"%s\",\"warps_per_block\":%d,\"handover\":%d,"
                 "\"heavy_min_p\":%d,\"heavy_heat\":%d,\"ms\":%.6g}",
                 first ? "" : ",", kv.first.c_str(), kv.second.version.c_str(),
                 kv.second.c.warps_per_block, kv.second.c.handover, kv.second.c.heavy_min_p,
                 kv.second.c.heavy_heat, (double)kv.second.c.ms);
        out += buf;
        first = false;
    }
    out += "}}\n";
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return SPMESL_EINVAL;
    const bool ok = fwrite(out.data(), 1, out.size(), f) == out.size();
    if (fclose(f) != 0 || !ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return SPMESL_EINVAL;
    }
    return SPMESL_OK;
}

}  // extern "C"
