// bs_tune.cu -- the autotuner's cache of chosen kernel variants (host code).
//
// An entry maps a tuning key -- GPU name and SM count, precision, tet rule, near rule, number of
// directions, the problem's size class (ceil(log2) of the evaluation points and of the tets), and whether
// the points are the mesh's nodes evaluated by bs_velocity_nodes (where the mesh walk can take the near
// field) or arbitrary points -- to
// the variant bs_autotune timed fastest, with that variant's launch shape as a check: an entry whose
// shape no longer matches the compiled variant table is ignored.  Entries are read from two JSON
// files: the one shipped beside the package (tune_cache.json next to the library's _build directory)
// and the file named by the environment variable BS_TUNE_CACHE (its entries take precedence).
// bs_autotune writes new entries to BS_TUNE_CACHE when it is set, else to the shipped file.
//
// The file holds one JSON object: {"libbs_tune_cache": 1, "entries": {"<key>": {"variant": v,
// "shape": "<shape>", "ms": t, "candidates": n}, ...}} with one entry per line (the reader scans for
// that line form only; anything else in the file is ignored).
#include <dlfcn.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "bs_internal.cuh"

namespace bs {
namespace {

struct Entry {
    int variant = -1;
    std::string shape;
    double ms = 0.0;
    int candidates = 0;
};

std::mutex g_mu;
bool g_loaded = false;
std::map<std::string, Entry> g_entries;

std::string library_dir()
{
    Dl_info info;
    if (dladdr(reinterpret_cast<void *>(&library_dir), &info) == 0 || !info.dli_fname) return ".";
    std::string p = info.dli_fname;
    const size_t s = p.find_last_of('/');
    return s == std::string::npos ? std::string(".") : p.substr(0, s);
}

std::string shipped_path() { return library_dir() + "/../tune_cache.json"; }

std::string user_path()
{
    const char *e = getenv("BS_TUNE_CACHE");
    return (e && *e) ? std::string(e) : std::string();
}

// the value of "name": in an entry line, as text (a number or a quoted string without the quotes)
bool field(const std::string &line, const char *name, std::string &out)
{
    const std::string tag = std::string("\"") + name + "\":";
    size_t p = line.find(tag);
    if (p == std::string::npos) return false;
    p += tag.size();
    while (p < line.size() && line[p] == ' ') ++p;
    if (p < line.size() && line[p] == '"') {
        const size_t q = line.find('"', p + 1);
        if (q == std::string::npos) return false;
        out = line.substr(p + 1, q - p - 1);
        return true;
    }
    size_t q = p;
    while (q < line.size() && line[q] != ',' && line[q] != '}') ++q;
    out = line.substr(p, q - p);
    return !out.empty();
}

void read_file(const std::string &path, std::map<std::string, Entry> &into)
{
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return;
    std::string line;
    char buf[1024];
    while (fgets(buf, sizeof buf, f)) {
        line += buf;
        if (line.empty() || line.back() != '\n') continue;  // a long line: keep reading
        // entry lines: "<key>": {"variant": v, "shape": "...", ...}
        const size_t k0 = line.find('"');
        const size_t k1 = k0 == std::string::npos ? k0 : line.find("\": {\"variant\"", k0 + 1);
        if (k1 != std::string::npos) {
            Entry e;
            std::string v, s, ms, c;
            if (field(line, "variant", v) && field(line, "shape", s)) {
                e.variant = atoi(v.c_str());
                e.shape = s;
                if (field(line, "ms", ms)) e.ms = atof(ms.c_str());
                if (field(line, "candidates", c)) e.candidates = atoi(c.c_str());
                into[line.substr(k0 + 1, k1 - k0 - 1)] = e;
            }
        }
        line.clear();
    }
    fclose(f);
}

void load_locked()
{
    if (g_loaded) return;
    read_file(shipped_path(), g_entries);
    const std::string u = user_path();
    if (!u.empty()) read_file(u, g_entries);  // later entries replace earlier ones
    g_loaded = true;
}

bool write_file(const std::string &path, const std::map<std::string, Entry> &entries)
{
    const std::string tmp = path + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return false;
    fprintf(f, "{\"libbs_tune_cache\": 1, \"entries\": {\n");
    size_t i = 0;
    for (const auto &kv : entries) {
        fprintf(f, "\"%s\": {\"variant\": %d, \"shape\": \"%s\", \"ms\": %.4f, \"candidates\": %d}%s\n",
                kv.first.c_str(), kv.second.variant, kv.second.shape.c_str(), kv.second.ms, kv.second.candidates,
                ++i < entries.size() ? "," : "");
    }
    fprintf(f, "}}\n");
    const bool ok = fclose(f) == 0;
    return ok && rename(tmp.c_str(), path.c_str()) == 0;
}

int ceil_log2(int64_t n)
{
    int b = 0;
    while (b < 62 && ((int64_t)1 << b) < n) ++b;
    return b;
}

}  // namespace

std::string variant_shape_string(int precision, int Q, int near_rule, int variant)
{
    const VariantList vl = velocity_variants(precision, Q, near_rule);
    if (variant < 0 || variant >= vl.n) return std::string();
    const VariantShape &s = vl.v[variant].s;
    char b[96];
    snprintf(b, sizeof b, "P%d T%d S%d B%d D%d U%d %s J%d", s.P, s.TILE, s.S, s.MINB, s.DR, s.U, s.PK ? "pp" : "qp",
             s.UJ);
    return b;
}

std::string tune_key(const char *gpu_name, int n_sm, int precision, int Q, int near_rule, int L, int64_t k,
                     int64_t n_tets, bool at_nodes)
{
    char b[256];
    snprintf(b, sizeof b, "%s/%dsm %s q%d %s L%d k2^%d t2^%d %s", gpu_name, n_sm,
             precision == BS_FP32 ? "fp32" : "fp64", Q, near_rule == BS_NEAR_EXACT ? "exact" : "ray", L,
             ceil_log2(k), ceil_log2(n_tets), at_nodes ? "nodes" : "points");
    return b;
}

int tune_lookup(const std::string &key, int precision, int Q, int near_rule)
{
    std::lock_guard<std::mutex> lock(g_mu);
    load_locked();
    const auto it = g_entries.find(key);
    if (it == g_entries.end()) return -1;
    const Entry &e = it->second;
    if (e.shape != variant_shape_string(precision, Q, near_rule, e.variant)) return -1;  // written by a library with another variant table
    return e.variant;
}

bool tune_store(const std::string &key, int precision, int Q, int near_rule, int variant, double ms, int candidates)
{
    std::lock_guard<std::mutex> lock(g_mu);
    load_locked();
    Entry e;
    e.variant = variant;
    e.shape = variant_shape_string(precision, Q, near_rule, variant);
    e.ms = ms;
    e.candidates = candidates;
    g_entries[key] = e;
    // the target file gets its own entries plus this one (entries read from the other file stay there)
    const std::string u = user_path();
    const std::string path = u.empty() ? shipped_path() : u;
    std::map<std::string, Entry> file;
    read_file(path, file);
    file[key] = e;
    return write_file(path, file);
}

}  // namespace bs
