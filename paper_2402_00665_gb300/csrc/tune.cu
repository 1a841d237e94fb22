// tune.cu -- the autotuner's choices and their cache (host code).
//
// A choice is made for one configuration: the GPU, the size bucket of the
// trees (ceil(log2 n)), the Morton bits, the primitive kind, the query kind
// (-1 for the sort of a build) and the number of trees built together (1 for
// a single tree, the instance count of a batch). It records the sort's tile
// shape and ranking (a variant of sort.cu's table; for a single tree's codes
// wider than 30 bits, also whether the top-bits sort takes one pass fewer)
// and how the collecting walk runs (one thread per query in CTAs of 256 or
// 512 threads, or groups of 8, 16 or 32 lanes, and the query order's Morton
// bits), each with the time it measured. lbvh_tree_autotune and the batch path fill the
// cache by timing every candidate on the caller's own data; builds and
// queries look their configuration up and fall back to the defaults. The
// cache can be written to and read from a small JSON file, so a process can
// start with the choices an earlier one measured.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "lbvh_internal.cuh"

namespace lbvh {

namespace {

std::mutex g_mu;
std::map<TuneKey, TuneChoice> g_cache;

bool key_less(const TuneKey &a, const TuneKey &b) {
    return std::tie(a.gpu, a.n_log2, a.bits, a.kind, a.qkind, a.instances) <
           std::tie(b.gpu, b.n_log2, b.bits, b.kind, b.qkind, b.instances);
}

}  // namespace

bool TuneKey::operator<(const TuneKey &o) const { return key_less(*this, o); }

int ceil_log2(int64_t x) {
    int k = 0;
    while (k < 62 && (int64_t(1) << k) < x) ++k;
    return k;
}

std::string current_gpu_name() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return "unknown";
    static std::mutex mu;
    static std::map<int, std::string> names;
    std::lock_guard<std::mutex> lock(mu);
    auto it = names.find(dev);
    if (it != names.end()) return it->second;
    cudaDeviceProp p{};
    std::string name = cudaGetDeviceProperties(&p, dev) == cudaSuccess ? std::string(p.name) : "unknown";
    names[dev] = name;
    return name;
}

TuneKey tune_key(int64_t n, int bits, int kind, int qkind, int64_t instances) {
    return TuneKey{current_gpu_name(), ceil_log2(n), bits, kind, qkind, instances};
}

bool tune_find(const TuneKey &k, TuneChoice *out) {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_cache.find(k);
    if (it == g_cache.end()) return false;
    *out = it->second;
    return true;
}

void tune_put(const TuneKey &k, const TuneChoice &c) {
    std::lock_guard<std::mutex> lock(g_mu);
    TuneChoice &e = g_cache[k];
    if (c.sort >= 0) {
        e.sort = c.sort;
        e.sort_ms = c.sort_ms;
    }
    if (c.walk >= 0) {
        e.walk = c.walk;
        e.walk_ms = c.walk_ms;
    }
}

int tune_sort_choice(int64_t n, int bits, int kind, int64_t instances) {
    TuneChoice c;
    return tune_find(tune_key(n, bits, kind, -1, instances), &c) ? c.sort : -1;
}

int tune_walk_choice(int64_t n, int bits, int kind, int qkind, int64_t instances) {
    TuneChoice c;
    return tune_find(tune_key(n, bits, kind, qkind, instances), &c) && c.walk >= 0 ? c.walk : kWalkThread;
}

namespace {

// ---- a reader for the flat JSON this file writes: an "entries" array of
// objects whose values are strings (no escapes but \" and \\) or numbers.

struct Reader {
    const char *p, *end;
    void ws() {
        while (p < end && (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t')) ++p;
    }
    bool eat(char c) {
        ws();
        if (p < end && *p == c) {
            ++p;
            return true;
        }
        return false;
    }
    bool str(std::string *out) {
        ws();
        if (p >= end || *p != '"') return false;
        ++p;
        out->clear();
        while (p < end && *p != '"') {
            if (*p == '\\' && p + 1 < end) ++p;
            out->push_back(*p++);
        }
        if (p >= end) return false;
        ++p;
        return true;
    }
    bool num(double *out) {
        ws();
        char *e = nullptr;
        const std::string s(p, (size_t)std::min<ptrdiff_t>(end - p, 64));
        *out = std::strtod(s.c_str(), &e);
        if (e == s.c_str()) return false;
        p += e - s.c_str();
        return true;
    }
};

bool parse_entry(Reader &r, TuneKey *k, TuneChoice *c) {
    if (!r.eat('{')) return false;
    bool have_gpu = false;
    while (true) {
        std::string name;
        if (!r.str(&name) || !r.eat(':')) return false;
        if (name == "gpu") {
            if (!r.str(&k->gpu)) return false;
            have_gpu = true;
        } else {
            double v = 0;
            if (!r.num(&v)) return false;
            if (name == "n_log2") k->n_log2 = (int)v;
            else if (name == "bits") k->bits = (int)v;
            else if (name == "kind") k->kind = (int)v;
            else if (name == "qkind") k->qkind = (int)v;
            else if (name == "instances") k->instances = (int64_t)v;
            else if (name == "sort_variant") c->sort = (int)v;
            else if (name == "sort_ms") c->sort_ms = (float)v;
            else if (name == "walk_variant") c->walk = (int)v;
            else if (name == "walk_ms") c->walk_ms = (float)v;
        }
        if (r.eat(',')) continue;
        if (r.eat('}')) return have_gpu;
        return false;
    }
}

}  // namespace

}  // namespace lbvh

extern "C" {

lbvh_status lbvh_tune_save(const char *path) {
    if (!path) return LBVH_ERR_INVALID;
    std::vector<std::pair<lbvh::TuneKey, lbvh::TuneChoice>> all;
    {
        std::lock_guard<std::mutex> lock(lbvh::g_mu);
        all.assign(lbvh::g_cache.begin(), lbvh::g_cache.end());
    }
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return LBVH_ERR_INVALID;
    std::fprintf(f, "{\"lbvh_tune_cache\": 1, \"entries\": [");
    for (size_t i = 0; i < all.size(); ++i) {
        const auto &k = all[i].first;
        const auto &c = all[i].second;
        std::string gpu;
        for (char ch : k.gpu) {
            if (ch == '"' || ch == '\\') gpu.push_back('\\');
            gpu.push_back(ch);
        }
        std::fprintf(f,
                     "%s\n  {\"gpu\": \"%s\", \"n_log2\": %d, \"bits\": %d, \"kind\": %d, \"qkind\": %d, "
                     "\"instances\": %lld, \"sort_variant\": %d, \"sort_ms\": %.4f, \"walk_variant\": %d, "
                     "\"walk_ms\": %.4f}",
                     i ? "," : "", gpu.c_str(), k.n_log2, k.bits, k.kind, k.qkind, (long long)k.instances, c.sort,
                     c.sort_ms, c.walk, c.walk_ms);
    }
    std::fprintf(f, "\n]}\n");
    const bool ok = std::fclose(f) == 0;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return LBVH_ERR_INVALID;
    }
    return LBVH_OK;
}

lbvh_status lbvh_tune_load(const char *path) {
    if (!path) return LBVH_ERR_INVALID;
    FILE *f = std::fopen(path, "rb");
    if (!f) return LBVH_ERR_INVALID;
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    std::fclose(f);
    lbvh::Reader r{text.data(), text.data() + text.size()};
    const size_t at = text.find("\"entries\"");
    if (at == std::string::npos) return LBVH_ERR_INVALID;
    r.p = text.data() + at + 9;
    if (!r.eat(':') || !r.eat('[')) return LBVH_ERR_INVALID;
    std::vector<std::pair<lbvh::TuneKey, lbvh::TuneChoice>> got_entries;
    if (!r.eat(']')) {
        while (true) {
            lbvh::TuneKey k{};
            lbvh::TuneChoice c{};
            if (!lbvh::parse_entry(r, &k, &c)) return LBVH_ERR_INVALID;
            got_entries.emplace_back(k, c);
            if (r.eat(',')) continue;
            if (r.eat(']')) break;
            return LBVH_ERR_INVALID;
        }
    }
    for (auto &e : got_entries) {
        // a choice this build of the library does not have is dropped (a
        // batch's sort takes a tile shape alone, a single tree's build also
        // the top-bits pass count)
        const int sorts = e.first.instances > 1 ? lbvh::sort_variant_count() : lbvh::build_sort_choices();
        if (e.second.sort >= sorts) e.second.sort = -1;
        if (e.second.walk >= lbvh::kWalkChoices) e.second.walk = -1;
        lbvh::tune_put(e.first, e.second);
    }
    return LBVH_OK;
}

void lbvh_tune_clear(void) {
    std::lock_guard<std::mutex> lock(lbvh::g_mu);
    lbvh::g_cache.clear();
}

int lbvh_tune_entries(void) {
    std::lock_guard<std::mutex> lock(lbvh::g_mu);
    return (int)lbvh::g_cache.size();
}

int lbvh_sort_variant_count(void) { return lbvh::build_sort_choices(); }

int lbvh_walk_variant_count(void) { return lbvh::kWalkChoices; }

}  // extern "C"
