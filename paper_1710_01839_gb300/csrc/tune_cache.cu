// Persistent tuning cache (host code only).  The paper's Section 3 tuning
// takes hours per CPU (its Tables 2 and 4), which is why it predicts block
// times from reduced runs; on the GPU a tuning run takes seconds, but it is
// still worth doing once per problem shape and device rather than once per
// process.  The cache is an append-only text file with one JSON object per
// line:
//
//   {"v":1,"t":"meas",   <key>, "algo":..,"n_min":..,"depth":..,"rows":..,"reps":..,"ms":..}
//   {"v":1,"t":"choice", <key>, "algo":..,"n_min":..,"depth":..,"best_ms":.., <report fields>}
//   <key> = "dev":"<device name>","ver":<library version>,"sms":..,"kind":..,"bits":..,"m":..,"l":..,"n":..
//
// Every timing the tuner takes is appended (and flushed) as soon as it is
// measured, so a tuning run that is killed resumes without timing again what
// it had finished; a finished run appends its choice, which MPGEMM_AUTO then
// uses (in this and in later processes that open the file) before the cost
// model.  Lines that do not parse (a line cut short by a kill, damage) are
// skipped and counted; records of another device name, SM count or library
// version are kept in the file but not used.
#include <fcntl.h>
#include <unistd.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "tune.h"

namespace mpg {

namespace {

struct JVal {
    enum Kind { NUM, STR, ARR, NUL } kind = NUL;
    double num = 0;
    std::string str;
    std::vector<double> arr;
};
using JObj = std::map<std::string, JVal>;

struct Parser {
    const char* p;
    const char* e;
    void ws() {
        while (p < e && (*p == ' ' || *p == '\t' || *p == '\r' || *p == '\n')) p++;
    }
    bool lit(char c) {
        ws();
        if (p < e && *p == c) {
            p++;
            return true;
        }
        return false;
    }
    bool str(std::string* out) {
        ws();
        if (p >= e || *p != '"') return false;
        p++;
        out->clear();
        while (p < e && *p != '"') {
            if (*p == '\\' || (unsigned char)*p < 0x20) return false;   // the writer never escapes
            out->push_back(*p++);
        }
        if (p >= e) return false;
        p++;
        return true;
    }
    bool num(double* out) {
        ws();
        if (p + 4 <= e && !strncmp(p, "null", 4)) {
            p += 4;
            *out = NAN;
            return true;
        }
        char buf[64];
        int k = 0;
        while (p < e && k < 63 && (strchr("0123456789+-.eE", *p) != nullptr)) buf[k++] = *p++;
        if (k == 0) return false;
        buf[k] = 0;
        char* end = nullptr;
        *out = strtod(buf, &end);
        return end == buf + k;
    }
    bool value(JVal* v) {
        ws();
        if (p < e && *p == '"') {
            v->kind = JVal::STR;
            return str(&v->str);
        }
        if (p < e && *p == '[') {
            p++;
            v->kind = JVal::ARR;
            if (lit(']')) return true;
            for (;;) {
                double x;
                if (!num(&x)) return false;
                v->arr.push_back(x);
                if (lit(']')) return true;
                if (!lit(',')) return false;
            }
        }
        v->kind = JVal::NUM;
        return num(&v->num);
    }
    bool object(JObj* o) {
        if (!lit('{')) return false;
        if (lit('}')) return true;
        for (;;) {
            std::string k;
            JVal v;
            if (!str(&k) || !lit(':') || !value(&v)) return false;
            (*o)[k] = v;
            if (lit('}')) break;
            if (!lit(',')) return false;
        }
        ws();
        return p == e;
    }
};

bool get_num(const JObj& o, const char* k, double* x) {
    auto it = o.find(k);
    if (it == o.end() || it->second.kind != JVal::NUM) return false;
    *x = it->second.num;
    return true;
}

bool get_int(const JObj& o, const char* k, int64_t* x) {
    double d;
    if (!get_num(o, k, &d) || std::isnan(d) || d != std::floor(d) || std::fabs(d) > 9.0e15) return false;
    *x = (int64_t)d;
    return true;
}

bool get_arr(const JObj& o, const char* k, size_t len, double* out) {
    auto it = o.find(k);
    if (it == o.end() || it->second.kind != JVal::ARR || it->second.arr.size() != len) return false;
    for (size_t i = 0; i < len; i++) out[i] = it->second.arr[i];
    return true;
}

// (kind, bits, m, l, n, sms)
using PKey = std::tuple<int, int, int64_t, int64_t, int64_t, int>;
// (algo, n_min, depth, rows, reps)
using MKey = std::tuple<int, int, int, int64_t, int>;

struct Cache {
    std::mutex mu;
    int fd = -1;
    std::string path;
    std::map<PKey, std::map<MKey, double>> meas;
    std::map<PKey, mpgemm_tune_report> choices;
    int n_meas = 0, n_choice = 0, n_skipped = 0, n_foreign = 0;
};

Cache& cache() {
    static Cache c;
    return c;
}

std::string device_name() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();   // a host without a GPU: every record of this process says so
        return "none";
    }
    std::string s(prop.name);
    for (char& ch : s)
        if (ch == '"' || ch == '\\' || (unsigned char)ch < 0x20) ch = '_';
    return s;
}

const std::string& this_device() {
    static std::string name = device_name();
    return name;
}

std::string key_json(const PKey& k) {
    char buf[512];
    snprintf(buf, sizeof buf, "\"dev\":\"%s\",\"ver\":%d,\"sms\":%d,\"kind\":%d,\"bits\":%d,\"m\":%lld,\"l\":%lld,\"n\":%lld",
             this_device().c_str(), mpgemm_version(), std::get<5>(k), std::get<0>(k), std::get<1>(k),
             (long long)std::get<2>(k), (long long)std::get<3>(k), (long long)std::get<4>(k));
    return buf;
}

std::string num_json(double x) {
    if (std::isnan(x) || std::isinf(x)) return "null";
    char buf[40];
    snprintf(buf, sizeof buf, "%.17g", x);
    return buf;
}

template <class T>
std::string arr_json(const T* a, int len) {
    std::string s = "[";
    for (int i = 0; i < len; i++) {
        if (i) s += ",";
        s += num_json((double)a[i]);
    }
    return s + "]";
}

// Whole lines with one write(2) on an O_APPEND descriptor: concurrent writers
// do not interleave within a line.
void append_line(Cache& c, const std::string& line) {
    if (c.fd < 0) return;
    std::string s = line + "\n";
    const char* p = s.data();
    size_t left = s.size();
    while (left > 0) {
        ssize_t w = write(c.fd, p, left);
        if (w <= 0) return;
        p += w;
        left -= (size_t)w;
    }
}

bool parse_key(const JObj& o, PKey* k, bool* ours) {
    int64_t ver, sms, kind, bits, m, l, n;
    auto dv = o.find("dev");
    if (dv == o.end() || dv->second.kind != JVal::STR) return false;
    if (!get_int(o, "ver", &ver) || !get_int(o, "sms", &sms) || !get_int(o, "kind", &kind) ||
        !get_int(o, "bits", &bits) || !get_int(o, "m", &m) || !get_int(o, "l", &l) || !get_int(o, "n", &n))
        return false;
    *k = PKey((int)kind, (int)bits, m, l, n, (int)sms);
    *ours = dv->second.str == this_device() && ver == mpgemm_version();
    return true;
}

bool parse_choice(const JObj& o, mpgemm_tune_report* r) {
    int64_t algo, n_min, depth, n_cand;
    memset(r, 0, sizeof *r);
    if (!get_int(o, "algo", &algo) || !get_int(o, "n_min", &n_min) || !get_int(o, "depth", &depth) ||
        !get_num(o, "best_ms", &r->best_ms) || !get_int(o, "n_cand", &n_cand) || n_cand < 0 || n_cand > 8)
        return false;
    if (algo < MPGEMM_SIMPLE || algo > MPGEMM_STRASSEN || depth < 0 || depth > 4 || n_min < 1 || n_min > 1024)
        return false;
    r->algo = (int)algo;
    r->n_min = (int)n_min;
    r->depth = (int)depth;
    r->n_cand = (int)n_cand;
    double cn[8], cr[8];
    if (!get_arr(o, "cand_n_min", (size_t)n_cand, cn) || !get_arr(o, "cand_rows", (size_t)n_cand, cr) ||
        !get_arr(o, "cand_sample_ms", (size_t)n_cand, r->cand_sample_ms) ||
        !get_arr(o, "cand_pred_ms", (size_t)n_cand, r->cand_pred_ms) ||
        !get_arr(o, "cand_full_ms", (size_t)n_cand, r->cand_full_ms) || !get_num(o, "simple_ms", &r->simple_ms) ||
        !get_num(o, "block_ms", &r->block_ms) || !get_arr(o, "strassen_ms", 5, r->strassen_ms))
        return false;
    for (int i = 0; i < n_cand; i++) {
        r->cand_n_min[i] = (int)cn[i];
        r->cand_rows[i] = (int64_t)cr[i];
    }
    return true;
}

void load_line(Cache& c, const char* b, const char* e) {
    while (b < e && (*b == ' ' || *b == '\t' || *b == '\r')) b++;
    if (b == e) return;
    JObj o;
    Parser ps{b, e};
    double v;
    auto t = o.end();
    if (!ps.object(&o) || !get_num(o, "v", &v) || v != 1.0 || (t = o.find("t")) == o.end() ||
        t->second.kind != JVal::STR) {
        c.n_skipped++;
        return;
    }
    PKey k;
    bool ours = false;
    if (!parse_key(o, &k, &ours)) {
        c.n_skipped++;
        return;
    }
    if (t->second.str == "meas") {
        int64_t algo, n_min, depth, rows, reps;
        double ms;
        if (!get_int(o, "algo", &algo) || !get_int(o, "n_min", &n_min) || !get_int(o, "depth", &depth) ||
            !get_int(o, "rows", &rows) || !get_int(o, "reps", &reps) || !get_num(o, "ms", &ms) ||
            !(ms >= 0.0)) {
            c.n_skipped++;
            return;
        }
        if (!ours) {
            c.n_foreign++;
            return;
        }
        c.meas[k][MKey((int)algo, (int)n_min, (int)depth, rows, (int)reps)] = ms;
        c.n_meas++;
    } else if (t->second.str == "choice") {
        mpgemm_tune_report r;
        if (!parse_choice(o, &r)) {
            c.n_skipped++;
            return;
        }
        if (!ours) {
            c.n_foreign++;
            return;
        }
        c.choices[k] = r;
        c.n_choice++;
        remember_choice(std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k),
                        std::get<5>(k), Choice{r.algo, r.n_min, r.depth});
    } else {
        c.n_skipped++;
    }
}

PKey pkey(const TuneKey& k) { return PKey(k.kind, k.bits, k.m, k.l, k.n, k.sms); }

}  // namespace

bool tune_cache_lookup_meas(const TuneKey& k, int algo, int n_min, int depth, int64_t rows, int reps, double* ms) {
    Cache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    if (c.fd < 0) return false;
    auto it = c.meas.find(pkey(k));
    if (it == c.meas.end()) return false;
    auto jt = it->second.find(MKey(algo, n_min, depth, rows, reps));
    if (jt == it->second.end()) return false;
    *ms = jt->second;
    return true;
}

void tune_cache_append_meas(const TuneKey& k, int algo, int n_min, int depth, int64_t rows, int reps, double ms) {
    Cache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    if (c.fd < 0) return;
    const PKey pk = pkey(k);
    c.meas[pk][MKey(algo, n_min, depth, rows, reps)] = ms;
    char buf[160];
    snprintf(buf, sizeof buf, ",\"algo\":%d,\"n_min\":%d,\"depth\":%d,\"rows\":%lld,\"reps\":%d,\"ms\":", algo, n_min,
             depth, (long long)rows, reps);
    append_line(c, "{\"v\":1,\"t\":\"meas\"," + key_json(pk) + buf + num_json(ms) + "}");
}

bool tune_cache_lookup_choice(const TuneKey& k, mpgemm_tune_report* rep) {
    Cache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    if (c.fd < 0) return false;
    auto it = c.choices.find(pkey(k));
    if (it == c.choices.end()) return false;
    *rep = it->second;
    return true;
}

void tune_cache_append_choice(const TuneKey& k, const mpgemm_tune_report* r) {
    Cache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    if (c.fd < 0) return;
    const PKey pk = pkey(k);
    c.choices[pk] = *r;
    char buf[160];
    snprintf(buf, sizeof buf, ",\"algo\":%d,\"n_min\":%d,\"depth\":%d,\"n_cand\":%d,\"best_ms\":", r->algo, r->n_min,
             r->depth, r->n_cand);
    std::string s = "{\"v\":1,\"t\":\"choice\"," + key_json(pk) + buf + num_json(r->best_ms);
    s += ",\"cand_n_min\":" + arr_json(r->cand_n_min, r->n_cand);
    s += ",\"cand_rows\":" + arr_json(r->cand_rows, r->n_cand);
    s += ",\"cand_sample_ms\":" + arr_json(r->cand_sample_ms, r->n_cand);
    s += ",\"cand_pred_ms\":" + arr_json(r->cand_pred_ms, r->n_cand);
    s += ",\"cand_full_ms\":" + arr_json(r->cand_full_ms, r->n_cand);
    s += ",\"simple_ms\":" + num_json(r->simple_ms) + ",\"block_ms\":" + num_json(r->block_ms);
    s += ",\"strassen_ms\":" + arr_json(r->strassen_ms, 5) + "}";
    append_line(c, s);
}

}  // namespace mpg

using namespace mpg;

extern "C" {

int mpgemm_tune_cache_open(const char* path) {
    Cache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    if (c.fd >= 0) {
        close(c.fd);
        c.fd = -1;
    }
    c.meas.clear();
    c.choices.clear();
    c.n_meas = c.n_choice = c.n_skipped = c.n_foreign = 0;
    c.path.clear();
    if (!path) return MPGEMM_OK;
    if (!*path) return MPGEMM_EINVAL;
    int fd = open(path, O_RDWR | O_APPEND | O_CREAT | O_CLOEXEC, 0644);
    if (fd < 0) return MPGEMM_EINVAL;
    // read what is there; a last line without its newline is a cut-short
    // write and is skipped (and made a line of its own before appending)
    std::string data;
    char buf[1 << 16];
    ssize_t r;
    lseek(fd, 0, SEEK_SET);
    while ((r = read(fd, buf, sizeof buf)) > 0) data.append(buf, (size_t)r);
    if (r < 0) {
        close(fd);
        return MPGEMM_EINVAL;
    }
    size_t pos = 0;
    while (pos < data.size()) {
        size_t nl = data.find('\n', pos);
        if (nl == std::string::npos) {
            c.n_skipped++;
            break;
        }
        load_line(c, data.data() + pos, data.data() + nl);
        pos = nl + 1;
    }
    c.fd = fd;
    c.path = path;
    if (!data.empty() && data.back() != '\n') append_line(c, "");
    return MPGEMM_OK;
}

int mpgemm_tune_cache_stats(int* choices, int* measurements, int* skipped_lines, int* foreign_records) {
    Cache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    if (choices) *choices = c.n_choice;
    if (measurements) *measurements = c.n_meas;
    if (skipped_lines) *skipped_lines = c.n_skipped;
    if (foreign_records) *foreign_records = c.n_foreign;
    return c.fd >= 0 ? 1 : 0;
}

}  // extern "C"
