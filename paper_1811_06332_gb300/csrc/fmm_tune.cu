// Persistent cache of autotuned kernel shapes: a small JSON object in a
// file, one entry per key (GPU name, order, basis, precision form, depth),
//   {
//    "NVIDIA GB300|p=8|basis=1|prec=3|depth=6": {"kernel": 0, "cw": 48, "niss": 4, "ms": 2.581},
//    ...
//   }
// Reading tolerates a missing or malformed file (no entry); writing replaces
// the entry of its key and rewrites the file through a temporary name.
#include <sys/stat.h>

#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "fmm_internal.h"

namespace fmm {

struct TuneEntry {
    std::string key;
    int kernel = 0, cw = 0, niss = 0;
    double ms = 0.0;
};

static std::string json_escape(const std::string& s) {
    std::string o;
    for (char c : s) {
        if (c == '"' || c == '\\') {
            o += '\\';
            o += c;
        } else if ((unsigned char)c < 0x20) {
            o += ' ';
        } else {
            o += c;
        }
    }
    return o;
}

// Parses a JSON string starting at s[i] == '"'; on success i is past it.
static bool parse_string(const std::string& s, size_t& i, std::string& out) {
    if (i >= s.size() || s[i] != '"') return false;
    out.clear();
    for (++i; i < s.size(); ++i) {
        if (s[i] == '\\') {
            if (++i >= s.size()) return false;
            out += s[i];
        } else if (s[i] == '"') {
            ++i;
            return true;
        } else {
            out += s[i];
        }
    }
    return false;
}

static void skip_ws(const std::string& s, size_t& i) {
    while (i < s.size() && (s[i] == ' ' || s[i] == '\n' || s[i] == '\r' || s[i] == '\t' || s[i] == ',')) ++i;
}

// Reads every well-formed entry; stops at the first malformed one.
static std::vector<TuneEntry> read_entries(const char* path) {
    std::vector<TuneEntry> v;
    FILE* f = fopen(path, "rb");
    if (!f) return v;
    std::string s;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof buf, f)) > 0 && s.size() < (1u << 22)) s.append(buf, n);
    fclose(f);
    size_t i = 0;
    skip_ws(s, i);
    if (i >= s.size() || s[i] != '{') return v;
    ++i;
    for (;;) {
        skip_ws(s, i);
        if (i >= s.size() || s[i] == '}') break;
        TuneEntry e;
        if (!parse_string(s, i, e.key)) break;
        skip_ws(s, i);
        if (i >= s.size() || s[i] != ':') break;
        ++i;
        skip_ws(s, i);
        if (i >= s.size() || s[i] != '{') break;
        const size_t end = s.find('}', i);
        if (end == std::string::npos) break;
        const std::string body = s.substr(i + 1, end - i - 1);
        i = end + 1;
        int seen = 0;
        size_t j = 0;
        for (;;) {
            skip_ws(body, j);
            std::string name;
            if (!parse_string(body, j, name)) break;
            skip_ws(body, j);
            if (j >= body.size() || body[j] != ':') break;
            ++j;
            char* endp = nullptr;
            const double val = strtod(body.c_str() + j, &endp);
            if (endp == body.c_str() + j) break;
            j = (size_t)(endp - body.c_str());
            if (name == "kernel") { e.kernel = (int)val; seen |= 1; }
            else if (name == "cw") { e.cw = (int)val; seen |= 2; }
            else if (name == "niss") { e.niss = (int)val; seen |= 4; }
            else if (name == "ms") { e.ms = val; seen |= 8; }
        }
        if (seen != 15) break;
        v.push_back(e);
    }
    return v;
}

int tune_cache_get(const char* path, const char* key, int* kernel, int* cw, int* niss, double* ms) {
    if (!path || !key) return -1;
    for (const TuneEntry& e : read_entries(path)) {
        if (e.key == key) {
            *kernel = e.kernel;
            *cw = e.cw;
            *niss = e.niss;
            if (ms) *ms = e.ms;
            return 1;
        }
    }
    return 0;
}

int tune_cache_put(const char* path, const char* key, int kernel, int cw, int niss, double ms) {
    if (!path || !key || !*path) return -1;
    std::vector<TuneEntry> v = read_entries(path);
    bool found = false;
    for (TuneEntry& e : v)
        if (e.key == key) {
            e.kernel = kernel; e.cw = cw; e.niss = niss; e.ms = ms;
            found = true;
        }
    if (!found) {
        TuneEntry e;
        e.key = key; e.kernel = kernel; e.cw = cw; e.niss = niss; e.ms = ms;
        v.push_back(e);
    }
    // create the file's directories (each prefix ending in '/')
    const std::string p(path);
    for (size_t k = p.find('/', 1); k != std::string::npos; k = p.find('/', k + 1)) {
        const std::string dir = p.substr(0, k);
        if (mkdir(dir.c_str(), 0755) != 0 && errno != EEXIST) return -2;
    }
    const std::string tmp = p + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return -2;
    fprintf(f, "{\n");
    for (size_t k = 0; k < v.size(); ++k)
        fprintf(f, " \"%s\": {\"kernel\": %d, \"cw\": %d, \"niss\": %d, \"ms\": %.4f}%s\n",
                json_escape(v[k].key).c_str(), v[k].kernel, v[k].cw, v[k].niss, v[k].ms,
                k + 1 < v.size() ? "," : "");
    fprintf(f, "}\n");
    const bool ok = fclose(f) == 0;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return -2;
    }
    return 0;
}

}  // namespace fmm
