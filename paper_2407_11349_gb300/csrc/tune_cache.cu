// Autotuner cache: a small JSON file that maps a configuration key to the
// tuned sweep configuration, so a process can skip the search on a device and
// problem shape it has tuned before.  Host code only.
//
// The file is written by this library as a JSON object with one entry per
// line:
//   {
//   "NVIDIA GB300|sm_103|single|n<=2^20|flags=0": {"variant": 0, "chunk": 16, "order": 0, "ms": 365.359, "nvariants": 5, "kc": 1},
//   ...
//   }
// The reader accepts exactly that shape and skips any line it cannot parse,
// so a damaged file degrades to cache misses, never to an error.  Entries
// written by a build with a different number of sweep variants are ignored.
// "kc" (chains per CTA of a batch's group sweep) may be absent, meaning 1.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

namespace hk {

int sweep_num_variants();

namespace {

struct Entry {
    std::string key;
    int variant = -1, chunk = 0, order = 0, nvariants = 0, kc = 1;
    double ms = 0.0;
};

bool key_ok(const char* key) {
    if (!key || !*key) return false;
    for (const char* c = key; *c; ++c)
        if (*c == '"' || *c == '\\' || *c == '\n' || *c == '\r' || static_cast<unsigned char>(*c) < 0x20)
            return false;
    return std::strlen(key) < 512;
}

// Value of "name": <number> inside [b, e), or false.
bool field(const char* b, const char* e, const char* name, double* out) {
    const std::string pat = std::string("\"") + name + "\"";
    const std::string s(b, e);
    const size_t k = s.find(pat);
    if (k == std::string::npos) return false;
    size_t i = k + pat.size();
    while (i < s.size() && (s[i] == ' ' || s[i] == '\t')) ++i;
    if (i >= s.size() || s[i] != ':') return false;
    ++i;
    const char* start = s.c_str() + i;
    char* end = nullptr;
    const double v = std::strtod(start, &end);
    if (end == start) return false;
    *out = v;
    return true;
}

// Parse one line of the file; false if it is not an entry.
bool parse_line(const std::string& line, Entry* e) {
    size_t i = line.find('"');
    if (i == std::string::npos) return false;
    const size_t j = line.find('"', i + 1);
    if (j == std::string::npos) return false;
    e->key = line.substr(i + 1, j - i - 1);
    const size_t ob = line.find('{', j), cb = line.find('}', j);
    if (ob == std::string::npos || cb == std::string::npos || cb < ob) return false;
    const char* b = line.c_str() + ob;
    const char* en = line.c_str() + cb;
    double v, c, o, ms, nv;
    if (!field(b, en, "variant", &v) || !field(b, en, "chunk", &c) || !field(b, en, "order", &o) ||
        !field(b, en, "ms", &ms) || !field(b, en, "nvariants", &nv))
        return false;
    for (double x : {v, c, o, nv})
        if (!(x >= -1e6 && x <= 1e6)) return false;  // also rejects NaN
    if (!std::isfinite(ms)) return false;
    e->variant = static_cast<int>(v);
    e->chunk = static_cast<int>(c);
    e->order = static_cast<int>(o);
    e->ms = ms;
    e->nvariants = static_cast<int>(nv);
    double kc = 1.0;
    if (field(b, en, "kc", &kc) && !(kc >= 1.0 && kc <= 64.0)) return false;
    e->kc = static_cast<int>(kc);
    return key_ok(e->key.c_str());
}

std::vector<Entry> read_all(const char* path) {
    std::vector<Entry> out;
    FILE* f = std::fopen(path, "rb");
    if (!f) return out;
    std::string line;
    int ch;
    while ((ch = std::fgetc(f)) != EOF) {
        if (ch == '\n') {
            Entry e;
            if (parse_line(line, &e)) out.push_back(e);
            line.clear();
        } else if (line.size() < 4096) {
            line.push_back(static_cast<char>(ch));
        }
    }
    Entry e;
    if (!line.empty() && parse_line(line, &e)) out.push_back(e);
    std::fclose(f);
    return out;
}

}  // namespace

// 1: found (outputs written), 0: absent, HAWKES_ERR_ARG: bad arguments.
int tune_cache_get(const char* path, const char* key, int* variant, int* chunk, int* order,
                   double* ms, int* kc) {
    if (!path || !key_ok(key)) return HAWKES_ERR_ARG;
    const int nv = sweep_num_variants();
    int found = 0;
    for (const Entry& e : read_all(path)) {
        if (e.key != key || e.nvariants != nv || e.variant < 0 || e.variant >= nv) continue;
        if (variant) *variant = e.variant;
        if (chunk) *chunk = e.chunk;
        if (order) *order = e.order;
        if (ms) *ms = e.ms;
        if (kc) *kc = e.kc;
        found = 1;  // the last valid entry for a key wins
    }
    return found;
}

// Insert or replace an entry; the file is rewritten through a temporary file
// and renamed into place, so readers never see a half-written file.
int tune_cache_put(const char* path, const char* key, int variant, int chunk, int order, double ms,
                   int kc) {
    if (!path || !key_ok(key) || variant < 0 || variant >= sweep_num_variants() || chunk < 0 ||
        order < 0 || !(ms >= 0.0) || kc < 1 || kc > 64)
        return HAWKES_ERR_ARG;
    std::vector<Entry> all = read_all(path);
    Entry n;
    n.key = key;
    n.variant = variant;
    n.chunk = chunk;
    n.order = order;
    n.ms = ms;
    n.nvariants = sweep_num_variants();
    n.kc = kc;
    bool replaced = false;
    for (Entry& e : all)
        if (e.key == n.key) {
            e = n;
            replaced = true;
        }
    if (!replaced) all.push_back(n);
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return HAWKES_ERR_IO;
    bool ok = std::fputs("{\n", f) >= 0;
    for (size_t k = 0; k < all.size() && ok; ++k) {
        const Entry& e = all[k];
        ok = std::fprintf(f,
                          "\"%s\": {\"variant\": %d, \"chunk\": %d, \"order\": %d, \"ms\": %.3f, "
                          "\"nvariants\": %d, \"kc\": %d}%s\n",
                          e.key.c_str(), e.variant, e.chunk, e.order, e.ms, e.nvariants, e.kc,
                          k + 1 < all.size() ? "," : "") > 0;
    }
    ok = ok && std::fputs("}\n", f) >= 0;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return HAWKES_ERR_IO;
    }
    return HAWKES_OK;
}

// Smallest power-of-two exponent e with 2^e >= v (v >= 1).
int log2_ceil(double v) {
    int e = 0;
    while (e < 120 && std::ldexp(1.0, e) < v) ++e;
    return e;
}

// "<device name>|sm_<cc>|" for the current device; empty on failure.
std::string device_key() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return std::string();
    std::string name(prop.name);
    for (char& c : name)
        if (c == '"' || c == '\\' || c == '|' || static_cast<unsigned char>(c) < 0x20) c = '_';
    char buf[64];
    std::snprintf(buf, sizeof(buf), "|sm_%d%d|", prop.major, prop.minor);
    return name + buf;
}

}  // namespace hk

extern "C" int hawkes_tune_cache_get(const char* cache_path, const char* key, int* variant,
                                     int* chunk, int* order, double* ms) {
    return hk::tune_cache_get(cache_path, key, variant, chunk, order, ms, nullptr);
}

extern "C" int hawkes_tune_cache_put(const char* cache_path, const char* key, int variant,
                                     int chunk, int order, double ms) {
    return hk::tune_cache_put(cache_path, key, variant, chunk, order, ms, 1);
}
