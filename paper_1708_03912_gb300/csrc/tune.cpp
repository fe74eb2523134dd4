// Tuning table of launch shapes: a process-wide list of (kernel, shape key) ->
// (two integer parameters, measured time), filled by the autotuners (fl_tune_*),
// consulted by the solvers when the caller leaves a launch parameter at 0, and
// persisted as a small JSON file.  Entries carry the device name they were measured
// on; a file from another device contributes nothing.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "context.h"

namespace fl {

struct TuneEntry {
    std::string device, kernel;
    int64_t n;
    int nrhs, nslices, p0, p1;
    double ms;
};

static std::mutex g_tune_mu;
static std::vector<TuneEntry> g_tune;
static std::atomic<unsigned> g_tune_gen{0};  // bumped on every change of the table

unsigned tune_generation() { return g_tune_gen.load(std::memory_order_acquire); }

std::string device_name() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    return prop.name;
}

void tune_record(const std::string& device, const std::string& kernel, int64_t n, int nrhs, int nslices, int p0,
                 int p1, double ms) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_gen.fetch_add(1, std::memory_order_acq_rel);
    for (TuneEntry& e : g_tune) {
        if (e.device == device && e.kernel == kernel && e.n == n && e.nrhs == nrhs && e.nslices == nslices) {
            e.p0 = p0;
            e.p1 = p1;
            e.ms = ms;
            return;
        }
    }
    g_tune.push_back({device, kernel, n, nrhs, nslices, p0, p1, ms});
}

bool tune_lookup(const std::string& device, const std::string& kernel, int64_t n, int nrhs, int nslices, int* p0,
                 int* p1) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const TuneEntry& e : g_tune) {
        if (e.device == device && e.kernel == kernel && e.n == n && e.nrhs == nrhs && e.nslices == nslices) {
            *p0 = e.p0;
            *p1 = e.p1;
            return true;
        }
    }
    return false;
}

// -------------------------------------------------------------- JSON file --
// {"entries": [{"device": "...", "kernel": "...", "n": 1, "nrhs": 1, "nslices": 1,
//               "p0": 1, "p1": 1, "ms": 0.1}, ...]}
static std::string escape(const std::string& s) {
    std::string o;
    for (char c : s) {
        if (c == '"' || c == '\\') o += '\\';
        if ((unsigned char)c >= 0x20) o += c;
    }
    return o;
}

// minimal reader for the format above: string and number values of flat objects
struct Reader {
    const std::string& t;
    size_t i = 0;
    explicit Reader(const std::string& text) : t(text) {}
    void ws() {
        while (i < t.size() && (t[i] == ' ' || t[i] == '\n' || t[i] == '\r' || t[i] == '\t')) ++i;
    }
    bool eat(char c) {
        ws();
        if (i < t.size() && t[i] == c) {
            ++i;
            return true;
        }
        return false;
    }
    bool str(std::string& out) {
        ws();
        if (i >= t.size() || t[i] != '"') return false;
        ++i;
        out.clear();
        while (i < t.size() && t[i] != '"') {
            if (t[i] == '\\' && i + 1 < t.size()) ++i;
            out += t[i++];
        }
        if (i >= t.size()) return false;
        ++i;
        return true;
    }
    bool num(double& v) {
        ws();
        const char* b = t.c_str() + i;
        char* e = nullptr;
        v = std::strtod(b, &e);
        if (e == b) return false;
        i += (size_t)(e - b);
        return true;
    }
};

static bool parse(const std::string& text, std::vector<TuneEntry>& out) {
    Reader r(text);
    std::string key;
    if (!r.eat('{') || !r.str(key) || key != "entries" || !r.eat(':') || !r.eat('[')) return false;
    if (r.eat(']')) return r.eat('}');
    do {
        if (!r.eat('{')) return false;
        TuneEntry e{"", "", 0, 0, 0, 0, 0, 0.0};
        do {
            std::string k;
            if (!r.str(k) || !r.eat(':')) return false;
            if (k == "device" || k == "kernel") {
                std::string v;
                if (!r.str(v)) return false;
                (k == "device" ? e.device : e.kernel) = v;
            } else {
                double v;
                if (!r.num(v)) return false;
                if (k == "n") e.n = (int64_t)v;
                else if (k == "nrhs") e.nrhs = (int)v;
                else if (k == "nslices") e.nslices = (int)v;
                else if (k == "p0") e.p0 = (int)v;
                else if (k == "p1") e.p1 = (int)v;
                else if (k == "ms") e.ms = v;
            }
        } while (r.eat(','));
        if (!r.eat('}')) return false;
        out.push_back(e);
    } while (r.eat(','));
    return r.eat(']') && r.eat('}');
}

}  // namespace fl

using namespace fl;

extern "C" {

int fl_tune_record(const char* kernel, int64_t n, int nrhs, int nslices, int p0, int p1, double ms) {
    if (!kernel || !*kernel || n < 1) return FL_EINVAL;
    tune_record(device_name(), kernel, n, nrhs, nslices, p0, p1, ms);
    return FL_OK;
}

int fl_tune_lookup(const char* kernel, int64_t n, int nrhs, int nslices, int* p0, int* p1) {
    if (!kernel || !p0 || !p1) return FL_EINVAL;
    return tune_lookup(device_name(), kernel, n, nrhs, nslices, p0, p1) ? FL_OK : FL_ENOTIMPL;
}

void fl_tune_clear(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_gen.fetch_add(1, std::memory_order_acq_rel);
    g_tune.clear();
}

int fl_tune_count(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    return (int)g_tune.size();
}

int fl_tune_save(const char* path) {
    if (!path) return FL_EINVAL;
    FILE* f = std::fopen(path, "w");
    if (!f) return FL_EINVAL;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    std::fprintf(f, "{\"entries\": [");
    for (size_t k = 0; k < g_tune.size(); ++k) {
        const TuneEntry& e = g_tune[k];
        std::fprintf(f,
                     "%s\n  {\"device\": \"%s\", \"kernel\": \"%s\", \"n\": %lld, \"nrhs\": %d, \"nslices\": %d, "
                     "\"p0\": %d, \"p1\": %d, \"ms\": %.6g}",
                     k ? "," : "", escape(e.device).c_str(), escape(e.kernel).c_str(), (long long)e.n, e.nrhs,
                     e.nslices, e.p0, e.p1, e.ms);
    }
    std::fprintf(f, "\n]}\n");
    return std::fclose(f) == 0 ? FL_OK : FL_EINVAL;
}

int fl_tune_load(const char* path) {
    if (!path) return FL_EINVAL;
    FILE* f = std::fopen(path, "r");
    if (!f) return FL_EINVAL;
    std::string text;
    char buf[4096];
    size_t k;
    while ((k = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, k);
    std::fclose(f);
    std::vector<TuneEntry> entries;
    if (!parse(text, entries)) return FL_EINVAL;
    for (const TuneEntry& e : entries) tune_record(e.device, e.kernel, e.n, e.nrhs, e.nslices, e.p0, e.p1, e.ms);
    return FL_OK;
}

}  // extern "C"
