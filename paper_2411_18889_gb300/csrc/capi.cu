// capi.cu -- the C ABI declared in include/nbody.h: argument checks, the
// per-(device, stream) workspace cache, staging of host arrays, kernel-shape
// choice and the launch sequences of each call.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <dlfcn.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "nbody_internal.cuh"

namespace {

thread_local int t_last_cuda = 0;

int cuda_fail(cudaError_t e) {
    t_last_cuda = (int)e;
    if (e == cudaErrorMemoryAllocation) return NBODY_ENOMEM;
    return NBODY_ECUDA;
}
#define NB_CUDA(call)                               \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)
#define NB_CHECK(expr)           \
    do {                         \
        int r_ = (expr);         \
        if (r_ != NBODY_OK) return r_; \
    } while (0)

// Host-side fault injection for tests: NBODY_FAULT=alloc makes workspace
// allocation report NBODY_ENOMEM, NBODY_FAULT=launch makes the launch report
// NBODY_ECUDA, NBODY_FAULT=tune makes reading a kernel-shape table fail (the
// built-in table then serves).  Nothing is sent to the GPU in any case.
bool fault(const char* what) {
    const char* f = getenv("NBODY_FAULT");
    return f != nullptr && strcmp(f, what) == 0;
}


// ---------------------------------------------------------------------------
// Launch accounting and optional force-kernel timing (for benchmarks).
// ---------------------------------------------------------------------------
std::atomic<int64_t> g_launches{0};
std::atomic<bool> g_prof_on{false};
std::mutex g_prof_mu;
// Kernels timed by event pairs while profiling is on.
enum ProfKind { PROF_FORCE = 0, PROF_PACK = 1, PROF_KICK = 2, PROF_VJP = 3, PROF_KINDS = 4 };
struct ProfPair {
    cudaEvent_t a, b;
    int kind;
};
std::vector<ProfPair> g_prof_used, g_prof_free;
double g_prof_ms[PROF_KINDS] = {};
int64_t g_prof_n[PROF_KINDS] = {};

bool prof_pair(ProfPair* out, int kind = PROF_FORCE) {
    if (!g_prof_on.load()) return false;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfPair p;
    if (!g_prof_free.empty()) {
        p = g_prof_free.back();
        g_prof_free.pop_back();
    } else {
        if (cudaEventCreate(&p.a) != cudaSuccess) return false;
        if (cudaEventCreate(&p.b) != cudaSuccess) {
            cudaEventDestroy(p.a);
            return false;
        }
    }
    p.kind = kind;
    g_prof_used.push_back(p);
    *out = p;
    return true;
}

// Wait for every recorded pair and add its time to its kind (caller holds g_prof_mu).
cudaError_t prof_drain() {
    for (auto& p : g_prof_used) {
        cudaError_t e = cudaEventSynchronize(p.b);
        if (e != cudaSuccess) return e;
        float t = 0.0f;
        e = cudaEventElapsedTime(&t, p.a, p.b);
        if (e != cudaSuccess) return e;
        g_prof_ms[p.kind] += t;
        g_prof_n[p.kind] += 1;
        g_prof_free.push_back(p);
    }
    g_prof_used.clear();
    return cudaSuccess;
}

// A launch bracketed by an event pair of `kind` while profiling is on.
template <typename F>
cudaError_t timed(int kind, cudaStream_t st, F launch) {
    ProfPair pp;
    const bool on = prof_pair(&pp, kind);
    if (on) (void)cudaEventRecord(pp.a, st);
    const cudaError_t e = launch();
    if (on) (void)cudaEventRecord(pp.b, st);
    return e;
}

// Queue `launches` kernels' worth of accounting after a successful launch
// (while a graph is being captured the kernels are only recorded: they are
// counted when the graph runs).
thread_local bool t_capturing = false;
thread_local int t_captured = 0;
inline void count(int launches) {
    if (t_capturing)
        t_captured += launches;
    else
        g_launches += launches;
}

struct DeviceInfo {
    bool checked = false;
    bool ok = false;
    int num_sms = 0;
};
std::mutex g_dev_mu;
std::map<int, DeviceInfo> g_dev;

int device_check(int* dev_out, int* sms_out) {
    int dev = 0;
    NB_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DeviceInfo& d = g_dev[dev];
    if (!d.checked) {
        int major = 0, minor = 0, sms = 0;
        NB_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
        NB_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
        NB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        d.ok = (major == 10 && minor == 3);  // the library carries sm_103a code only
        d.num_sms = sms;
        d.checked = true;
    }
    if (!d.ok) return NBODY_ENOTSUP;
    *dev_out = dev;
    *sms_out = d.num_sms;
    return NBODY_OK;
}

// ---------------------------------------------------------------------------
// Workspace: device buffers reused across calls on one (device, stream).
// ---------------------------------------------------------------------------
struct Buf {
    void* p = nullptr;
    size_t cap = 0;
};

enum BufId {
    B_JDUP,
    B_CENTRES,
    B_PARTIAL,
    B_ACC,
    B_POT,
    B_RED,
    B_OUT9,
    B_ERR,
    B_BATCH,
    B_VJX,
    B_VJV,
    B_VJM,
    B_VJTAPE,
    B_VJ,
    B_VCENTRES,
    B_VPARTIAL,
    B_VG,
    B_VGM,
    B_SEGX,
    B_SEGV,
    B_IPACK,
    B_ICENTRES,
    B_PERM,
    B_ORDS,
    B_UNI,
    B_STAGE0,
    NBUF = B_STAGE0 + 8
};

struct Workspace {
    int device = 0;
    cudaStream_t stream = nullptr;
    Buf buf[NBUF];
    cudaStream_t aux = nullptr;  // second stream (adjoint replay), created on first use
    cudaEvent_t ev[5] = {};      // ordering events between the two streams
    uint64_t gen = 0;            // bumped whenever a buffer moves (invalidates cached graphs)
    cudaStream_t cap = nullptr;  // private stream that repeated calls are captured on
    std::map<std::vector<uint64_t>, struct GraphEntry*> graphs;
    uint64_t tick = 0;
};

struct GraphEntry {
    int seen = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
    uint64_t last = 0;
};

void drop_graph(GraphEntry* e) {
    if (e->exec) (void)cudaGraphExecDestroy(e->exec);
    if (e->graph) (void)cudaGraphDestroy(e->graph);
    delete e;
}

int ensure_aux(Workspace* w) {
    if (w->aux != nullptr) return NBODY_OK;
    NB_CUDA(cudaStreamCreateWithFlags(&w->aux, cudaStreamNonBlocking));
    for (auto& e : w->ev) NB_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return NBODY_OK;
}

std::mutex g_ws_mu;
std::map<std::pair<int, cudaStream_t>, Workspace*> g_ws;

Workspace* workspace(int dev, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    auto key = std::make_pair(dev, st);
    auto it = g_ws.find(key);
    if (it != g_ws.end()) return it->second;
    Workspace* w = new Workspace();
    w->device = dev;
    w->stream = st;
    g_ws[key] = w;
    return w;
}

// Make buffer `id` hold at least `bytes`; growing waits for the stream's
// queued work (which may still read the old buffer) before freeing it.
int ensure(Workspace* w, int id, size_t bytes, void** out) {
    if (fault("alloc")) return NBODY_ENOMEM;
    Buf& b = w->buf[id];
    if (bytes == 0) bytes = 16;
    if (b.cap < bytes) {
        if (b.p != nullptr) {
            NB_CUDA(cudaStreamSynchronize(w->stream));
            NB_CUDA(cudaFree(b.p));
            b.p = nullptr;
            b.cap = 0;
        }
        size_t sz = bytes + bytes / 8;
        sz = (sz + 255) & ~(size_t)255;
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, sz);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            t_last_cuda = (int)e;
            return NBODY_ENOMEM;
        }
        if (id == B_ERR) NB_CUDA(cudaMemset(p, 0, sz));
        b.p = p;
        b.cap = sz;
        ++w->gen;
    }
    *out = b.p;
    return NBODY_OK;
}

// ---------------------------------------------------------------------------
// Host arrays: detect, copy in, copy back.
// ---------------------------------------------------------------------------
bool is_host_ptr(const void* p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeUnregistered || a.type == cudaMemoryTypeHost;
}

struct Staging {
    struct Item {
        void* user;
        size_t bytes;
        bool in, out, host;
        void* dev;
    };
    Workspace* ws;
    std::vector<Item> items;
    bool any_host = false;
    explicit Staging(Workspace* w) : ws(w) {}
    void add(const void* p, size_t bytes, bool in, bool out) {
        items.push_back(Item{const_cast<void*>(p), bytes, in, out, false, const_cast<void*>(p)});
    }
    int prepare() {
        for (auto& it : items)
            if (it.user != nullptr) {
                it.host = is_host_ptr(it.user);
                any_host |= it.host;
            }
        if (!any_host) return NBODY_OK;
        int k = 0;
        for (auto& it : items) {
            if (it.user == nullptr || !it.host) continue;
            void* d = nullptr;
            NB_CHECK(ensure(ws, B_STAGE0 + k++, it.bytes, &d));
            it.dev = d;
            if (it.in) NB_CUDA(cudaMemcpyAsync(d, it.user, it.bytes, cudaMemcpyHostToDevice, ws->stream));
        }
        return NBODY_OK;
    }
    int finish() {
        if (!any_host) return NBODY_OK;
        for (auto& it : items)
            if (it.user != nullptr && it.host && it.out)
                NB_CUDA(cudaMemcpyAsync(it.user, it.dev, it.bytes, cudaMemcpyDeviceToHost, ws->stream));
        NB_CUDA(cudaStreamSynchronize(ws->stream));
        return NBODY_OK;
    }
    void* dev(int i) const { return items[i].dev; }
};

// ---------------------------------------------------------------------------
// Kernel-shape choice.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Kernel-shape table: rules "force <pot> <n_min> <shape>", "vjp <n_min>
// <shape>", "batched [<n_min>] <shape>" (n_min of a batched rule is compared
// with the batch's largest system) read from the tuner's file (NBODY_TUNE_FILE, or
// nbody_tune.txt beside the library); the rule with the largest n_min <= n
// wins.  Built-in defaults (measured on GB300) apply when no file is found.
// ---------------------------------------------------------------------------
struct TuneRule {
    int kind;  // 0 force, 1 vjp, 2 batched
    int pot;
    int64_t n_min;
    int shape;
};
std::mutex g_tune_mu;
std::vector<TuneRule> g_tune;
bool g_tune_loaded = false;

void tune_defaults(std::vector<TuneRule>& r) {
    r.clear();
    r.push_back({0, 0, 0, 3});
    r.push_back({0, 0, 2560, 4});
    r.push_back({0, 0, 10240, 2});
    r.push_back({0, 1, 0, 4});
    r.push_back({0, 1, 10240, 1});
    r.push_back({0, 1, 49152, 2});
    r.push_back({1, 0, 0, 3});
    r.push_back({1, 0, 2560, 2});
    r.push_back({1, 0, 49152, 0});
    r.push_back({2, 0, 0, 3});
    r.push_back({2, 0, 320, 2});
    r.push_back({2, 0, 763, 0});
}

int kind_shapes(int kind) {
    return kind == 0 ? nbk::force_num_shapes() : kind == 1 ? nbk::vjp_num_shapes() : nbk::batched_num_shapes();
}

// Parse a table file into `out`; returns the number of rules or NBODY_EINVAL.
int tune_parse(const char* path, std::vector<TuneRule>& out) {
    if (fault("tune")) return NBODY_EINVAL;
    FILE* f = fopen(path, "r");
    if (f == nullptr) return NBODY_EINVAL;
    char line[256];
    int bad = 0;
    out.clear();
    while (fgets(line, sizeof line, f) != nullptr) {
        char* s = line;
        while (*s == ' ' || *s == '\t') ++s;
        if (*s == '#' || *s == '\n' || *s == '\0') continue;
        char kind[16] = {0};
        long long a = 0, b = 0, d = 0;
        TuneRule r{};
        if (sscanf(s, "%15s", kind) != 1) {
            bad = 1;
            break;
        }
        if (strcmp(kind, "force") == 0 && sscanf(s, "%*s %lld %lld %lld", &a, &b, &d) == 3) {
            r = {0, (int)a, (int64_t)b, (int)d};
        } else if (strcmp(kind, "vjp") == 0 && sscanf(s, "%*s %lld %lld", &b, &d) == 2) {
            r = {1, 0, (int64_t)b, (int)d};
        } else if (strcmp(kind, "batched") == 0 && sscanf(s, "%*s %lld %lld", &b, &d) == 2) {
            r = {2, 0, (int64_t)b, (int)d};  // n_min = largest system of the batch
        } else if (strcmp(kind, "batched") == 0 && sscanf(s, "%*s %lld", &d) == 1) {
            r = {2, 0, 0, (int)d};
        } else {
            bad = 1;
            break;
        }
        if (r.pot < 0 || r.pot > 1 || r.n_min < 0 || r.shape < 0 || r.shape >= kind_shapes(r.kind)) {
            bad = 1;
            break;
        }
        out.push_back(r);
    }
    fclose(f);
    if (bad) {
        out.clear();
        return NBODY_EINVAL;
    }
    return (int)out.size();
}

std::string default_tune_path() {
    const char* env = getenv("NBODY_TUNE_FILE");
    if (env != nullptr) return std::string(env);
    Dl_info info;
    if (dladdr((void*)&tune_defaults, &info) != 0 && info.dli_fname != nullptr) {
        std::string p(info.dli_fname);
        const size_t k = p.find_last_of('/');
        return (k == std::string::npos ? std::string(".") : p.substr(0, k)) + "/nbody_tune.txt";
    }
    return std::string();
}

void tune_ensure_loaded() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tune_loaded) return;
    std::vector<TuneRule> r;
    const std::string p = default_tune_path();
    if (p.empty() || tune_parse(p.c_str(), r) <= 0) tune_defaults(r);
    g_tune = r;
    g_tune_loaded = true;
}

int tuned_shape(int kind, int64_t n, int pot) {
    tune_ensure_loaded();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    int best = -1;
    int64_t best_n = -1;
    for (const TuneRule& r : g_tune)
        if (r.kind == kind && (kind != 0 || r.pot == pot) && r.n_min <= n && r.n_min > best_n) {
            best = r.shape;
            best_n = r.n_min;
        }
    if (best < 0) {  // the file has no rule for this case: built-in default
        std::vector<TuneRule> d;
        tune_defaults(d);
        for (const TuneRule& r : d)
            if (r.kind == kind && (kind != 0 || r.pot == pot) && r.n_min <= n && r.n_min > best_n) {
                best = r.shape;
                best_n = r.n_min;
            }
    }
    return best < 0 ? 0 : best;
}

int choose_shape(int64_t n, bool pot) {
    const char* env = getenv("NBODY_SHAPE");
    if (env != nullptr) {
        int k = atoi(env);
        if (k >= 0 && k < nbk::force_num_shapes()) return k;
    }
    return tuned_shape(0, n, pot ? 1 : 0);
}

struct Opts {
    cudaStream_t stream = nullptr;
    int precision = NBODY_PREC_MIXED;
    int accumulate = NBODY_ACC_COMPENSATED;
    int config = -1;
};

// max_config: the number of shapes of the call's kernel (force shapes unless
// the call says otherwise; the batched calls have their own).
int read_opts(const nbody_opts* o, Opts* r, int max_config = -1) {
    if (o == nullptr) return NBODY_OK;
    if (o->precision != NBODY_PREC_MIXED && o->precision != NBODY_PREC_PLAIN &&
        o->precision != NBODY_PREC_MIXED_UNSORTED)
        return NBODY_EINVAL;
    if (o->accumulate != NBODY_ACC_COMPENSATED && o->accumulate != NBODY_ACC_FP32 &&
        o->accumulate != NBODY_ACC_KAHAN_PAIR)
        return NBODY_EINVAL;
    if (max_config < 0) max_config = nbk::force_num_shapes();
    if (o->config < -1 || o->config >= max_config) return NBODY_EINVAL;
    if (o->reserved != 0) return NBODY_EINVAL;
    r->stream = (cudaStream_t)o->stream;
    r->precision = o->precision;
    r->accumulate = o->accumulate;
    r->config = o->config;
    return NBODY_OK;
}

bool finite_nonneg(double x) { return isfinite(x) && x >= 0.0; }

// Kernel summation mode for an NBODY_ACC_* option: 0 one FP32 running sum,
// 1 per-tile FP32 folded by Kahan summation, 2 Kahan summation per pair.
int summation_mode(int accumulate) {
    switch (accumulate) {
        case NBODY_ACC_FP32: return 0;
        case NBODY_ACC_KAHAN_PAIR: return 2;
        default: return 1;
    }
}

// Everything one force evaluation needs, sized for n on this workspace.
struct ForcePlan {
    int shape;
    int block;
    int64_t npad;
    float* jdup;
    double* centres;
    double* chunks[2];  // 256-body chunk sums, alternately read and written by the packs of a leapfrog
    double* partial;
    int* err;
    int num_sms;
    int* perm = nullptr;            // spatial order of the bodies (mixed precision), or none
    void* order_scratch = nullptr;
    int* uni = nullptr;             // device word: all source masses equal (set by issue_uniform)
};

// The equal-mass check: when every source has the same mass the force
// kernels of the plan take the pair loop without m_j.  plan_uniform sizes the
// flag (outside any graph capture); issue_uniform queues the check, once per
// call (the masses do not change between the evaluations of a call).
int plan_uniform(Workspace* ws, ForcePlan* fp) {
    void* p;
    NB_CHECK(ensure(ws, B_UNI, sizeof(int), &p));
    fp->uni = (int*)p;
    return NBODY_OK;
}

int issue_uniform(const ForcePlan& fp, int64_t n, const float* mass, cudaStream_t st) {
    count(1);
    NB_CUDA(nbk::uniform_mass_flag(n, mass, fp.uni, st));
    return NBODY_OK;
}

// Buffers of the spatial order (mixed precision sorts the bodies along a
// Morton curve so that each cell is a compact region).
int plan_order(Workspace* ws, int64_t n, ForcePlan* fp) {
    void *p, *q;
    NB_CHECK(ensure(ws, B_PERM, (size_t)n * sizeof(int), &p));
    NB_CHECK(ensure(ws, B_ORDS, nbk::order_scratch_bytes(n), &q));
    fp->perm = (int*)p;
    fp->order_scratch = q;
    return NBODY_OK;
}

int issue_order(const ForcePlan& fp, int64_t n, const double* pos, cudaStream_t st) {
    count(14);
    NB_CUDA(nbk::spatial_order(n, pos, fp.perm, fp.order_scratch, st));
    return NBODY_OK;
}

bool sorted_mixed(int precision) { return precision == NBODY_PREC_MIXED; }

int plan_force(Workspace* ws, int64_t n, int shape, int num_sms, ForcePlan* fp) {
    fp->shape = shape;
    fp->block = nbk::force_shape(shape).block;
    const int64_t nblk = (n + fp->block - 1) / fp->block;
    fp->npad = nblk * fp->block;
    fp->num_sms = num_sms;
    void* p;
    NB_CHECK(ensure(ws, B_JDUP, (size_t)fp->npad * nbk::kJdupFloats * sizeof(float), &p));
    fp->jdup = (float*)p;
    const size_t ncen = nbk::pack_centre_doubles(fp->npad, fp->block);
    NB_CHECK(ensure(ws, B_CENTRES, (ncen + nbk::pack_chunk_doubles(fp->npad)) * sizeof(double), &p));
    fp->centres = (double*)p;
    fp->chunks[0] = fp->centres + (ncen - nbk::pack_chunk_doubles(fp->npad));  // where pack_f64 writes them
    fp->chunks[1] = fp->centres + ncen;
    NB_CHECK(ensure(ws, B_PARTIAL, nbk::force_partial_doubles(shape, num_sms) * sizeof(double), &p));
    fp->partial = (double*)p;
    NB_CHECK(ensure(ws, B_ERR, sizeof(int), &p));
    fp->err = (int*)p;
    return NBODY_OK;
}

// defer (optional): leave the split i-blocks' partial sums to the pack kernel
// that consumes this evaluation (no fixup launch); see nbk::SplitSums.
int run_force(const ForcePlan& fp, int64_t n, float eps2, bool mixed, int summation, float* acc, float* pot,
              cudaStream_t st, nbk::SplitSums* defer = nullptr) {
    if (fault("launch")) return NBODY_ECUDA;
    nbk::ForceArgs a;
    a.jdup = fp.jdup;
    a.centres = mixed ? fp.centres : nullptr;
    a.eps2 = eps2;
    a.n = n;
    a.npad = fp.npad;
    a.acc = acc;
    a.pot = pot;
    a.partial = fp.partial;
    a.err = fp.err;
    a.summation = summation;
    a.perm = fp.perm;
    a.uni = fp.uni;
    ProfPair pp;
    const bool timed = prof_pair(&pp);
    int launched = 0;
    cudaError_t e = nbk::force_launch(fp.shape, a, fp.num_sms, st, &launched, timed ? pp.a : nullptr,
                                      timed ? pp.b : nullptr, defer);
    count(launched);
    NB_CUDA(e);
    return NBODY_OK;
}

struct Ctx {
    int dev, sms;
    Opts o;
    Workspace* ws;
};

int begin(const nbody_opts* opts, Ctx* c, int max_config = -1) {
    NB_CHECK(read_opts(opts, &c->o, max_config));
    NB_CHECK(device_check(&c->dev, &c->sms));
    c->ws = workspace(c->dev, c->o.stream);
    return NBODY_OK;
}

int shape_for(const Ctx& c, int64_t n, bool pot) { return c.o.config >= 0 ? c.o.config : choose_shape(n, pot); }

int check_opts_only(const nbody_opts* opts, int max_config = -1) {
    Opts o;
    return read_opts(opts, &o, max_config);
}

// ---- force evaluation on device arrays ----
int accel_f64_dev(Ctx& c, int64_t n, const double* pos, const float* mass, double eps, float* acc, float* pot) {
    ForcePlan fp;
    NB_CHECK(plan_force(c.ws, n, shape_for(c, n, pot != nullptr), c.sms, &fp));
    const bool plain = c.o.precision == NBODY_PREC_PLAIN;
    if (sorted_mixed(c.o.precision)) {
        NB_CHECK(plan_order(c.ws, n, &fp));
        NB_CHECK(issue_order(fp, n, pos, c.o.stream));
    }
    NB_CHECK(plan_uniform(c.ws, &fp));
    NB_CHECK(issue_uniform(fp, n, mass, c.o.stream));
    count(nbk::pack_f64_launches(plain));
    NB_CUDA(nbk::pack_f64(n, fp.npad, fp.block, const_cast<double*>(pos), nullptr, nullptr, mass, 0.0, 0.0, plain,
                          fp.jdup, fp.centres, c.o.stream, fp.perm, fp.err));
    return run_force(fp, n, (float)(eps * eps), !plain, summation_mode(c.o.accumulate), acc, pot,
                     c.o.stream);
}

int accel_f32_dev(Ctx& c, int64_t n, const float* pos, const float* mass, float eps, float* acc, float* pot) {
    ForcePlan fp;
    NB_CHECK(plan_force(c.ws, n, shape_for(c, n, pot != nullptr), c.sms, &fp));
    NB_CHECK(plan_uniform(c.ws, &fp));
    NB_CHECK(issue_uniform(fp, n, mass, c.o.stream));
    count(1);
    NB_CUDA(nbk::pack_f32(n, fp.npad, const_cast<float*>(pos), nullptr, nullptr, mass, 0.0f, 0.0f, fp.jdup,
                          c.o.stream));
    return run_force(fp, n, eps * eps, false, summation_mode(c.o.accumulate), acc, pot, c.o.stream);
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void nbody_opts_default(nbody_opts* o) {
    if (o == nullptr) return;
    o->stream = nullptr;
    o->precision = NBODY_PREC_MIXED;
    o->accumulate = NBODY_ACC_COMPENSATED;
    o->config = -1;
    o->reserved = 0;
}

int nbody_version(void) { return 1 * 10000 + 0 * 100 + 0; }

int nbody_num_configs(void) { return nbk::force_num_shapes(); }

int nbody_num_batched_configs(void) { return nbk::batched_num_shapes(); }

int nbody_config_block(int k) {
    if (k < 0 || k >= nbk::force_num_shapes()) return 0;
    return nbk::force_shape(k).block;
}

const char* nbody_strerror(int code) {
    switch (code) {
        case NBODY_OK: return "success";
        case NBODY_EINVAL: return "invalid argument";
        case NBODY_ENOMEM: return "out of memory";
        case NBODY_ECUDA: return "CUDA runtime error";
        case NBODY_ETIMEOUT: return "bounded device wait expired";
        case NBODY_EBOUNDS: return "device index out of range (checked build)";
        case NBODY_ENOTSUP: return "unsupported device or option";
        default: return "unknown error code";
    }
}

int nbody_last_cuda_error(void) { return t_last_cuda; }

int nbody_accel(int64_t n, const double* pos, const float* mass, double eps, float* acc, float* pot,
                const nbody_opts* opts) {
    NB_RANGE("nbody_accel");
    if (n < 0 || !finite_nonneg(eps)) return NBODY_EINVAL;
    if (n > 0 && (pos == nullptr || mass == nullptr || acc == nullptr)) return NBODY_EINVAL;
    NB_CHECK(check_opts_only(opts));
    if (n == 0) return NBODY_OK;
    Ctx c;
    NB_CHECK(begin(opts, &c));
    Staging sg(c.ws);
    sg.add(pos, (size_t)n * 3 * sizeof(double), true, false);
    sg.add(mass, (size_t)n * sizeof(float), true, false);
    sg.add(acc, (size_t)n * 3 * sizeof(float), false, true);
    sg.add(pot, (size_t)n * sizeof(float), false, true);
    NB_CHECK(sg.prepare());
    NB_CHECK(accel_f64_dev(c, n, (const double*)sg.dev(0), (const float*)sg.dev(1), eps, (float*)sg.dev(2),
                           pot ? (float*)sg.dev(3) : nullptr));
    return sg.finish();
}

int nbody_accel_f32(int64_t n, const float* pos, const float* mass, float eps, float* acc, float* pot,
                    const nbody_opts* opts) {
    NB_RANGE("nbody_accel_f32");
    if (n < 0 || !finite_nonneg((double)eps)) return NBODY_EINVAL;
    if (n > 0 && (pos == nullptr || mass == nullptr || acc == nullptr)) return NBODY_EINVAL;
    NB_CHECK(check_opts_only(opts));
    if (n == 0) return NBODY_OK;
    Ctx c;
    NB_CHECK(begin(opts, &c));
    Staging sg(c.ws);
    sg.add(pos, (size_t)n * 3 * sizeof(float), true, false);
    sg.add(mass, (size_t)n * sizeof(float), true, false);
    sg.add(acc, (size_t)n * 3 * sizeof(float), false, true);
    sg.add(pot, (size_t)n * sizeof(float), false, true);
    NB_CHECK(sg.prepare());
    NB_CHECK(accel_f32_dev(c, n, (const float*)sg.dev(0), (const float*)sg.dev(1), eps, (float*)sg.dev(2),
                           pot ? (float*)sg.dev(3) : nullptr));
    return sg.finish();
}

}  // extern "C"

// The launch sequence of a leapfrog call (state type V: double or float).
template <typename V>
static int leapfrog_issue(int64_t n, V* x, V* v, const float* m, double eps, double dt, int64_t steps,
                          const ForcePlan& fp, float* a, bool plain, int comp, cudaStream_t st) {
    const bool f64 = sizeof(V) == sizeof(double);
    const float eps2 = f64 ? (float)(eps * eps) : (float)eps * (float)eps;
    if (f64 && fp.perm != nullptr) NB_CHECK(issue_order(fp, n, (const double*)x, st));  // order of the call
    NB_CHECK(issue_uniform(fp, n, m, st));
    count(f64 ? nbk::pack_f64_launches(plain) : 1);
    NB_CUDA(timed(PROF_PACK, st, [&] {
        return f64 ? nbk::pack_f64(n, fp.npad, fp.block, (double*)x, nullptr, nullptr, m, 0.0, 0.0, plain, fp.jdup,
                                   fp.centres, st, fp.perm, fp.err)
                   : nbk::pack_f32(n, fp.npad, (float*)x, nullptr, nullptr, m, 0.0f, 0.0f, fp.jdup, st);
    }));
    // Every evaluation but the last is consumed by the next step's pack
    // kernel, which adds the split i-blocks' partial sums itself.
    nbk::SplitSums ss;
    NB_CHECK(run_force(fp, n, eps2, f64 && !plain, comp, a, nullptr, st, steps > 0 ? &ss : nullptr));
    for (int64_t s = 0; s < steps; ++s) {
        const double kick = (s == 0) ? 0.5 * dt : dt;  // merged closing + opening half kicks
        count(1);
        NB_CUDA(timed(PROF_PACK, st, [&] {
            if (f64 && !plain)  // one kernel: cell centres from the previous step's chunk sums
                return nbk::pack_f64_lagged(n, fp.npad, fp.block, (double*)x, (double*)v, a, m, kick, dt, fp.jdup,
                                            fp.centres, fp.chunks[s & 1], fp.chunks[(s + 1) & 1], st, fp.perm,
                                            fp.err, &ss);
            return f64 ? nbk::pack_f64(n, fp.npad, fp.block, (double*)x, (double*)v, a, m, kick, dt, plain, fp.jdup,
                                       fp.centres, st, fp.perm, fp.err, &ss)
                       : nbk::pack_f32(n, fp.npad, (float*)x, (float*)v, a, m, (float)kick, (float)dt, fp.jdup, st,
                                       &ss);
        }));
        NB_CHECK(run_force(fp, n, eps2, f64 && !plain, comp, a, nullptr, st, s + 1 < steps ? &ss : nullptr));
    }
    count(1);
    NB_CUDA(timed(PROF_KICK, st, [&] {
        return f64 ? nbk::kick_f64(n, (double*)v, a, 0.5 * dt, st) : nbk::kick_f32(n, (float*)v, a, 0.5f * (float)dt, st);
    }));
    return NBODY_OK;
}

// A call repeated with the same arguments and workspace (the loop of a
// simulation) is captured, on its second occurrence, into a CUDA graph that
// later occurrences launch as one unit; the first occurrence runs directly.
// `key` names everything the launch sequence depends on besides the contents
// of the buffers it reads; issue(stream) queues that sequence.
template <typename F>
static int run_graphed(Ctx& c, std::vector<uint64_t> key, bool graphable, F issue) {
    cudaStream_t st = c.o.stream;
    // Direct launches while profiling, on request, or under an injected CUDA
    // tool (a profiler measures kernels one launch at a time).
    if (!graphable || g_prof_on.load() || getenv("NBODY_NO_GRAPH") != nullptr ||
        getenv("CUDA_INJECTION64_PATH") != nullptr)
        return issue(st);
    key.push_back(c.ws->gen);
    auto found = c.ws->graphs.find(key);
    if (found == c.ws->graphs.end()) {
        // keep at most 16 entries (captured or only seen) per workspace:
        // drop the least recently used before adding one
        if (c.ws->graphs.size() >= 16) {
            auto victim = c.ws->graphs.begin();
            for (auto it = c.ws->graphs.begin(); it != c.ws->graphs.end(); ++it)
                if (it->second->last < victim->second->last) victim = it;
            drop_graph(victim->second);
            c.ws->graphs.erase(victim);
        }
        found = c.ws->graphs.emplace(key, new GraphEntry()).first;
    }
    GraphEntry* ge = found->second;
    ge->last = ++c.ws->tick;
    if (ge->exec != nullptr) {
        NB_CUDA(cudaGraphLaunch(ge->exec, st));
        count(ge->kernels);
        return NBODY_OK;
    }
    if (ge->seen++ == 0) return issue(st);
    if (c.ws->cap == nullptr) NB_CUDA(cudaStreamCreateWithFlags(&c.ws->cap, cudaStreamNonBlocking));
    NB_CUDA(cudaStreamBeginCapture(c.ws->cap, cudaStreamCaptureModeThreadLocal));
    t_capturing = true;
    t_captured = 0;
    const int rc = issue(c.ws->cap);
    t_capturing = false;
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c.ws->cap, &graph);
    cudaGraphExec_t exec = nullptr;
    if (rc != NBODY_OK || ec != cudaSuccess || graph == nullptr ||
        cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        (void)cudaGetLastError();
        if (graph) (void)cudaGraphDestroy(graph);
        ge->seen = 1;  // try again next time; run this call directly
        return issue(st);
    }
    ge->graph = graph;
    ge->exec = exec;
    ge->kernels = t_captured;
    NB_CUDA(cudaGraphLaunch(exec, st));
    count(ge->kernels);
    return NBODY_OK;
}

static uint64_t bits_of(double x) {
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
}

template <typename V>
static int leapfrog_run(Ctx& c, int64_t n, V* x, V* v, const float* m, double eps, double dt, int64_t steps,
                        bool graphable) {
    ForcePlan fp;
    NB_CHECK(plan_force(c.ws, n, shape_for(c, n, false), c.sms, &fp));
    void* p;
    NB_CHECK(ensure(c.ws, B_ACC, (size_t)n * 3 * sizeof(float), &p));
    float* a = (float*)p;
    const bool plain = sizeof(V) == sizeof(float) || c.o.precision == NBODY_PREC_PLAIN;
    const int comp = summation_mode(c.o.accumulate);
    if (sizeof(V) == sizeof(double) && sorted_mixed(c.o.precision)) NB_CHECK(plan_order(c.ws, n, &fp));
    NB_CHECK(plan_uniform(c.ws, &fp));
    const std::vector<uint64_t> key = {1, (uint64_t)sizeof(V), (uint64_t)n, (uint64_t)steps, (uint64_t)(uintptr_t)x,
                                       (uint64_t)(uintptr_t)v, (uint64_t)(uintptr_t)m, bits_of(eps), bits_of(dt),
                                       (uint64_t)fp.shape, (uint64_t)plain, (uint64_t)comp,
                                       (uint64_t)(fp.perm != nullptr)};
    return run_graphed(c, key, graphable, [&](cudaStream_t s) {
        return leapfrog_issue<V>(n, x, v, m, eps, dt, steps, fp, a, plain, comp, s);
    });
}

extern "C" {

int nbody_leapfrog(int64_t n, double* pos, double* vel, const float* mass, double eps, double dt, int64_t steps,
                   const nbody_opts* opts) {
    NB_RANGE("nbody_leapfrog");
    if (n < 0 || steps < 0 || !finite_nonneg(eps) || !isfinite(dt)) return NBODY_EINVAL;
    if (n > 0 && (pos == nullptr || vel == nullptr || mass == nullptr)) return NBODY_EINVAL;
    NB_CHECK(check_opts_only(opts));
    if (n == 0 || steps == 0) return NBODY_OK;
    Ctx c;
    NB_CHECK(begin(opts, &c));
    Staging sg(c.ws);
    sg.add(pos, (size_t)n * 3 * sizeof(double), true, true);
    sg.add(vel, (size_t)n * 3 * sizeof(double), true, true);
    sg.add(mass, (size_t)n * sizeof(float), true, false);
    NB_CHECK(sg.prepare());
    NB_CHECK(leapfrog_run<double>(c, n, (double*)sg.dev(0), (double*)sg.dev(1), (const float*)sg.dev(2), eps, dt,
                                  steps, !sg.any_host));
    return sg.finish();
}

int nbody_leapfrog_f32(int64_t n, float* pos, float* vel, const float* mass, float eps, float dt, int64_t steps,
                       const nbody_opts* opts) {
    NB_RANGE("nbody_leapfrog_f32");
    if (n < 0 || steps < 0 || !finite_nonneg((double)eps) || !isfinite(dt)) return NBODY_EINVAL;
    if (n > 0 && (pos == nullptr || vel == nullptr || mass == nullptr)) return NBODY_EINVAL;
    NB_CHECK(check_opts_only(opts));
    if (n == 0 || steps == 0) return NBODY_OK;
    Ctx c;
    NB_CHECK(begin(opts, &c));
    Staging sg(c.ws);
    sg.add(pos, (size_t)n * 3 * sizeof(float), true, true);
    sg.add(vel, (size_t)n * 3 * sizeof(float), true, true);
    sg.add(mass, (size_t)n * sizeof(float), true, false);
    NB_CHECK(sg.prepare());
    NB_CHECK(leapfrog_run<float>(c, n, (float*)sg.dev(0), (float*)sg.dev(1), (const float*)sg.dev(2), (double)eps,
                                 (double)dt, steps, !sg.any_host));
    return sg.finish();
}

// ---------------------------------------------------------------------------
// Separate sinks and sources
// ---------------------------------------------------------------------------
static int accel_ij_common(int64_t ni, const void* ipos, int64_t nj, const void* jpos, const float* jmass, double eps,
                           float* acc, float* pot, const nbody_opts* opts, bool f64) {
    if (ni < 0 || nj < 0 || !finite_nonneg(eps)) return NBODY_EINVAL;
    if (ni > 0 && (ipos == nullptr || acc == nullptr)) return NBODY_EINVAL;
    if (nj > 0 && (jpos == nullptr || jmass == nullptr)) return NBODY_EINVAL;
    NB_CHECK(check_opts_only(opts));
    if (ni == 0) return NBODY_OK;
    Ctx c;
    NB_CHECK(begin(opts, &c));
    cudaStream_t st = c.o.stream;
    if (nj == 0) {  // no sources: zero force and potential
        Staging sg(c.ws);
        sg.add(acc, (size_t)ni * 3 * sizeof(float), false, true);
        sg.add(pot, (size_t)ni * sizeof(float), false, true);
        NB_CHECK(sg.prepare());
        NB_CUDA(cudaMemsetAsync(sg.dev(0), 0, (size_t)ni * 3 * sizeof(float), st));
        if (pot) NB_CUDA(cudaMemsetAsync(sg.dev(1), 0, (size_t)ni * sizeof(float), st));
        return sg.finish();
    }
    const size_t vb = f64 ? sizeof(double) : sizeof(float);
    Staging sg(c.ws);
    sg.add(ipos, (size_t)ni * 3 * vb, true, false);
    sg.add(jpos, (size_t)nj * 3 * vb, true, false);
    sg.add(jmass, (size_t)nj * sizeof(float), true, false);
    sg.add(acc, (size_t)ni * 3 * sizeof(float), false, true);
    sg.add(pot, (size_t)ni * sizeof(float), false, true);
    NB_CHECK(sg.prepare());
    // shape from the larger side; both sides padded to whole cells of it
    ForcePlan fp;
    NB_CHECK(plan_force(c.ws, nj, shape_for(c, ni > nj ? ni : nj, pot != nullptr), c.sms, &fp));
    const int64_t niblk = (ni + fp.block - 1) / fp.block;
    const int64_t nipad = niblk * fp.block;
    void *pi, *pc;
    NB_CHECK(ensure(c.ws, B_IPACK, (size_t)nipad * nbk::kJdupFloats * sizeof(float), &pi));
    NB_CHECK(ensure(c.ws, B_ICENTRES, nbk::pack_centre_doubles(nipad, fp.block) * sizeof(double), &pc));
    const bool plain = !f64 || c.o.precision == NBODY_PREC_PLAIN;
    // sinks need no mass: pack them with the sources' first mass pointer unused
    if (f64) {
        count(2 * nbk::pack_f64_launches(plain));
        NB_CUDA(nbk::pack_f64(ni, nipad, fp.block, (double*)sg.dev(0), nullptr, nullptr, nullptr, 0.0, 0.0, plain,
                              (float*)pi, (double*)pc, st));
        NB_CUDA(nbk::pack_f64(nj, fp.npad, fp.block, (double*)sg.dev(1), nullptr, nullptr, (const float*)sg.dev(2),
                              0.0, 0.0, plain, fp.jdup, fp.centres, st));
    } else {
        count(2);
        NB_CUDA(nbk::pack_f32(ni, nipad, (float*)sg.dev(0), nullptr, nullptr, nullptr, 0.0f, 0.0f, (float*)pi, st));
        NB_CUDA(nbk::pack_f32(nj, fp.npad, (float*)sg.dev(1), nullptr, nullptr, (const float*)sg.dev(2), 0.0f, 0.0f,
                              fp.jdup, st));
    }
    NB_CHECK(plan_uniform(c.ws, &fp));
    NB_CHECK(issue_uniform(fp, nj, (const float*)sg.dev(2), st));
    if (fault("launch")) return NBODY_ECUDA;
    nbk::ForceArgs a;
    a.jdup = fp.jdup;
    a.centres = plain ? nullptr : fp.centres;
    a.eps2 = f64 ? (float)(eps * eps) : (float)eps * (float)eps;
    a.uni = fp.uni;
    a.n = ni;
    a.npad = fp.npad;
    a.ipack = (const float*)pi;
    a.icentres = plain ? nullptr : (const double*)pc;
    a.nipad = nipad;
    a.acc = (float*)sg.dev(3);
    a.pot = pot ? (float*)sg.dev(4) : nullptr;
    a.partial = fp.partial;
    a.err = fp.err;
    a.summation = summation_mode(c.o.accumulate);
    int launched = 0;
    cudaError_t e = nbk::force_launch(fp.shape, a, fp.num_sms, st, &launched);
    count(launched);
    NB_CUDA(e);
    return sg.finish();
}

int nbody_accel_ij(int64_t ni, const double* ipos, int64_t nj, const double* jpos, const float* jmass, double eps,
                   float* acc, float* pot, const nbody_opts* opts) {
    NB_RANGE("nbody_accel_ij");
    return accel_ij_common(ni, ipos, nj, jpos, jmass, eps, acc, pot, opts, true);
}

int nbody_accel_ij_f32(int64_t ni, const float* ipos, int64_t nj, const float* jpos, const float* jmass, float eps,
                       float* acc, float* pot, const nbody_opts* opts) {
    NB_RANGE("nbody_accel_ij_f32");
    return accel_ij_common(ni, ipos, nj, jpos, jmass, (double)eps, acc, pot, opts, false);
}

// ---------------------------------------------------------------------------
// Reverse mode
// ---------------------------------------------------------------------------
static int choose_vjp_shape(int64_t n) { return tuned_shape(1, n, 0); }

struct VjpPlan {
    int shape, block;
    int64_t npad;
    float* jv;
    double* centres;
    double* chunks[2];  // 256-body chunk sums, alternately read and written by the packs of the sweep
    double* partial;
    int* err;
    int* uni = nullptr;  // device word: all masses equal (the flag of the call's force plan)
};

static int plan_vjp(Workspace* ws, int64_t n, int shape, int num_sms, VjpPlan* vp) {
    vp->shape = shape;
    vp->block = nbk::vjp_shape(shape).block;
    const int64_t nblk = (n + vp->block - 1) / vp->block;
    vp->npad = nblk * vp->block;
    void* p;
    NB_CHECK(ensure(ws, B_VJ, (size_t)vp->npad * nbk::vjp_floats_per_body() * sizeof(float), &p));
    vp->jv = (float*)p;
    const size_t ncen = nbk::pack_centre_doubles(vp->npad, vp->block);
    NB_CHECK(ensure(ws, B_VCENTRES, (ncen + nbk::pack_chunk_doubles(vp->npad)) * sizeof(double), &p));
    vp->centres = (double*)p;
    vp->chunks[0] = vp->centres + (ncen - nbk::pack_chunk_doubles(vp->npad));  // where pack_vjp writes them
    vp->chunks[1] = vp->centres + ncen;
    NB_CHECK(ensure(ws, B_VPARTIAL, nbk::vjp_partial_doubles(shape, num_sms) * sizeof(double), &p));
    vp->partial = (double*)p;
    NB_CHECK(ensure(ws, B_ERR, sizeof(int), &p));
    vp->err = (int*)p;
    return NBODY_OK;
}

// defer (optional): leave the split blocks' partials to the next pack_vjp.
// acc (optional): also the force at the same positions (defer_acc: deferred).
static int run_vjp(const VjpPlan& vp, int64_t n, float eps2, bool mixed, bool has_mu, float* g_pos, float* g_mass,
                   int num_sms, cudaStream_t st, nbk::SplitSums* defer = nullptr, float* acc = nullptr,
                   nbk::SplitSums* defer_acc = nullptr) {
    if (fault("launch")) return NBODY_ECUDA;
    nbk::VjpArgs a;
    a.jv = vp.jv;
    a.centres = mixed ? vp.centres : nullptr;
    a.eps2 = eps2;
    a.n = n;
    a.npad = vp.npad;
    a.has_mu = has_mu;
    a.g_pos = g_pos;
    a.g_mass = g_mass;
    a.partial = vp.partial;
    a.err = vp.err;
    a.uni = vp.uni;
    a.acc = acc;
    int launched = 0;
    ProfPair pp;
    const bool timed_vjp = prof_pair(&pp, PROF_VJP);
    cudaError_t e = nbk::vjp_launch(vp.shape, a, num_sms, st, &launched, timed_vjp ? pp.a : nullptr,
                                    timed_vjp ? pp.b : nullptr, defer, defer_acc);
    count(launched);
    NB_CUDA(e);
    return NBODY_OK;
}

int nbody_accel_vjp(int64_t n, const double* pos, const float* mass, double eps, const float* g_acc,
                    const float* g_pot, float* g_pos, float* g_mass, const nbody_opts* opts) {
    NB_RANGE("nbody_accel_vjp");
    if (n < 0 || !finite_nonneg(eps)) return NBODY_EINVAL;
    if (n > 0 && (pos == nullptr || mass == nullptr || g_acc == nullptr || g_pos == nullptr || g_mass == nullptr))
        return NBODY_EINVAL;
    NB_CHECK(check_opts_only(opts));
    if (opts != nullptr && opts->config >= nbk::vjp_num_shapes()) return NBODY_EINVAL;
    if (n == 0) return NBODY_OK;
    Ctx c;
    NB_CHECK(begin(opts, &c));
    Staging sg(c.ws);
    sg.add(pos, (size_t)n * 3 * sizeof(double), true, false);
    sg.add(mass, (size_t)n * sizeof(float), true, false);
    sg.add(g_acc, (size_t)n * 3 * sizeof(float), true, false);
    sg.add(g_pot, (size_t)n * sizeof(float), true, false);
    sg.add(g_pos, (size_t)n * 3 * sizeof(float), false, true);
    sg.add(g_mass, (size_t)n * sizeof(float), false, true);
    NB_CHECK(sg.prepare());
    VjpPlan vp;
    NB_CHECK(plan_vjp(c.ws, n, c.o.config >= 0 ? c.o.config : choose_vjp_shape(n), c.sms, &vp));
    const bool plain = c.o.precision == NBODY_PREC_PLAIN;
    {
        void* pu;
        NB_CHECK(ensure(c.ws, B_UNI, sizeof(int), &pu));
        vp.uni = (int*)pu;
        count(1);
        NB_CUDA(nbk::uniform_mass_flag(n, (const float*)sg.dev(1), vp.uni, c.o.stream));
    }
    count(2);
    NB_CUDA(nbk::pack_vjp(n, vp.npad, vp.block, (const double*)sg.dev(0), (const float*)sg.dev(1),
                          (const float*)sg.dev(2), nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, 1.0,
                          g_pot ? (const float*)sg.dev(3) : nullptr, plain, vp.jv, vp.centres, c.o.stream));
    NB_CHECK(run_vjp(vp, n, (float)(eps * eps), !plain, g_pot != nullptr, (float*)sg.dev(4), (float*)sg.dev(5), c.sms,
                     c.o.stream));
    return sg.finish();
}

// Tape of a recorded leapfrog: for each checkpoint k = 0, c, 2c, ... < steps the
// positions x_k and the half-step velocity v_{k+1/2} (FP64 [n][3] each), then
// the final positions x_steps and the last half-step velocity v_{steps-1/2}.
int64_t nbody_tape_bytes(int64_t n, int64_t steps, int64_t ckpt_every) {
    if (n < 0 || steps < 0 || ckpt_every < 1) return -1;
    const int64_t nck = (steps + ckpt_every - 1) / ckpt_every;
    return (nck * 2 + 2) * n * 3 * (int64_t)sizeof(double);
}

static bool device_only(const void* p) { return p != nullptr && !is_host_ptr(p); }

int nbody_leapfrog_record(int64_t n, double* pos, double* vel, const float* mass, double eps, double dt,
                          int64_t steps, int64_t ckpt_every, void* tape, const nbody_opts* opts) {
    NB_RANGE("nbody_leapfrog_record");
    if (n < 0 || steps < 0 || ckpt_every < 1 || !finite_nonneg(eps) || !isfinite(dt)) return NBODY_EINVAL;
    if (n > 0 && (pos == nullptr || vel == nullptr || mass == nullptr || tape == nullptr)) return NBODY_EINVAL;
    NB_CHECK(check_opts_only(opts));
    if (n == 0) return NBODY_OK;
    Ctx c;
    NB_CHECK(begin(opts, &c));
    if (!device_only(pos) || !device_only(vel) || !device_only(mass) || !device_only(tape)) return NBODY_EINVAL;
    cudaStream_t st = c.o.stream;
    const size_t n3b = (size_t)n * 3 * sizeof(double);
    double* tp = (double*)tape;
    const int64_t nck = (steps + ckpt_every - 1) / ckpt_every;
    double* xK = tp + (size_t)nck * 2 * n * 3;
    if (steps == 0) {
        NB_CUDA(cudaMemcpyAsync(xK, pos, n3b, cudaMemcpyDeviceToDevice, st));
        return NBODY_OK;
    }
    ForcePlan fp;
    NB_CHECK(plan_force(c.ws, n, shape_for(c, n, false), c.sms, &fp));
    void* p;
    NB_CHECK(ensure(c.ws, B_ACC, (size_t)n * 3 * sizeof(float), &p));
    float* a = (float*)p;
    const bool plain = c.o.precision == NBODY_PREC_PLAIN;
    const int comp = summation_mode(c.o.accumulate);
    const float eps2 = (float)(eps * eps);
    if (sorted_mixed(c.o.precision)) {  // the same order nbody_leapfrog takes (from x_0)
        NB_CHECK(plan_order(c.ws, n, &fp));
        NB_CHECK(issue_order(fp, n, pos, st));
    }
    NB_CHECK(plan_uniform(c.ws, &fp));
    NB_CHECK(issue_uniform(fp, n, mass, st));
    count(nbk::pack_f64_launches(plain));
    NB_CUDA(nbk::pack_f64(n, fp.npad, fp.block, pos, nullptr, nullptr, mass, 0.0, 0.0, plain, fp.jdup, fp.centres,
                          st, fp.perm, fp.err));
    nbk::SplitSums ss;  // as nbody_leapfrog: the next pack adds the split blocks' partials
    NB_CHECK(run_force(fp, n, eps2, !plain, comp, a, nullptr, st, &ss));
    for (int64_t s = 0; s < steps; ++s) {
        const bool ck = (s % ckpt_every) == 0;
        double* slot = tp + (size_t)(s / ckpt_every) * 2 * n * 3;
        if (ck) NB_CUDA(cudaMemcpyAsync(slot, pos, n3b, cudaMemcpyDeviceToDevice, st));
        const double kick = (s == 0) ? 0.5 * dt : dt;
        count(1);
        if (plain)
            NB_CUDA(nbk::pack_f64(n, fp.npad, fp.block, pos, vel, a, mass, kick, dt, plain, fp.jdup, fp.centres, st,
                                  fp.perm, fp.err, &ss));
        else  // as nbody_leapfrog: one kernel, centres from the previous step's chunk sums
            NB_CUDA(nbk::pack_f64_lagged(n, fp.npad, fp.block, pos, vel, a, mass, kick, dt, fp.jdup, fp.centres,
                                         fp.chunks[s & 1], fp.chunks[(s + 1) & 1], st, fp.perm, fp.err, &ss));
        if (ck) NB_CUDA(cudaMemcpyAsync(slot + (size_t)n * 3, vel, n3b, cudaMemcpyDeviceToDevice, st));
        NB_CHECK(run_force(fp, n, eps2, !plain, comp, a, nullptr, st, s + 1 < steps ? &ss : nullptr));
    }
    NB_CUDA(cudaMemcpyAsync(xK + (size_t)n * 3, vel, n3b, cudaMemcpyDeviceToDevice, st));  // v_{K-1/2}
    count(1);
    NB_CUDA(nbk::kick_f64(n, vel, a, 0.5 * dt, st));
    NB_CUDA(cudaMemcpyAsync(xK, pos, n3b, cudaMemcpyDeviceToDevice, st));
    return NBODY_OK;
}

int nbody_leapfrog_vjp_tape(int64_t n, const float* mass, double eps, double dt, int64_t steps, int64_t ckpt_every,
                            const void* tape, const double* g_posT, const double* g_velT, double* g_pos0,
                            double* g_vel0, double* g_mass, const nbody_opts* opts) {
    NB_RANGE("nbody_leapfrog_vjp_tape");
    if (n < 0 || steps < 0 || ckpt_every < 1 || !finite_nonneg(eps) || !isfinite(dt)) return NBODY_EINVAL;
    if (n > 0 && (mass == nullptr || tape == nullptr || g_posT == nullptr || g_velT == nullptr ||
                  g_pos0 == nullptr || g_vel0 == nullptr || g_mass == nullptr))
        return NBODY_EINVAL;
    NB_CHECK(check_opts_only(opts));
    if (n == 0) return NBODY_OK;
    Ctx c;
    NB_CHECK(begin(opts, &c));
    if (!device_only(tape) || !device_only(mass)) return NBODY_EINVAL;
    cudaStream_t st = c.o.stream;
    const size_t n3b = (size_t)n * 3 * sizeof(double);
    Staging sg(c.ws);
    sg.add(g_posT, n3b, true, false);
    sg.add(g_velT, n3b, true, false);
    sg.add(g_pos0, n3b, false, true);
    sg.add(g_vel0, n3b, false, true);
    sg.add(g_mass, (size_t)n * sizeof(double), false, true);
    NB_CHECK(sg.prepare());
    double* lamx = (double*)sg.dev(2);
    double* lamv = (double*)sg.dev(3);
    double* gm_acc = (double*)sg.dev(4);
    NB_CUDA(cudaMemcpyAsync(lamx, sg.dev(0), n3b, cudaMemcpyDeviceToDevice, st));
    NB_CUDA(cudaMemcpyAsync(lamv, sg.dev(1), n3b, cudaMemcpyDeviceToDevice, st));
    NB_CUDA(cudaMemsetAsync(gm_acc, 0, (size_t)n * sizeof(double), st));
    if (steps == 0) return sg.finish();

    const bool plain = c.o.precision == NBODY_PREC_PLAIN;
    const float eps2 = (float)(eps * eps);
    const double h = 0.5 * dt;
    const double* tp = (const double*)tape;
    const int64_t nck = (steps + ckpt_every - 1) / ckpt_every;
    const double* xK = tp + (size_t)nck * 2 * n * 3;
    const double* vK = xK + (size_t)n * 3;  // v_{K-1/2}
    VjpPlan vp;
    NB_CHECK(plan_vjp(c.ws, n, choose_vjp_shape(n), c.sms, &vp));
    void *pg, *pgm, *pa, *px, *pv, *pu;
    NB_CHECK(ensure(c.ws, B_VG, (size_t)n * 3 * sizeof(float), &pg));
    NB_CHECK(ensure(c.ws, B_VGM, (size_t)n * sizeof(float), &pgm));
    NB_CHECK(ensure(c.ws, B_ACC, (size_t)n * 3 * sizeof(float), &pa));
    NB_CHECK(ensure(c.ws, B_SEGX, n3b, &px));
    NB_CHECK(ensure(c.ws, B_SEGV, n3b, &pv));
    NB_CHECK(ensure(c.ws, B_UNI, sizeof(int), &pu));
    float* g = (float*)pg;
    float* gm = (float*)pgm;
    float* a = (float*)pa;
    double* X = (double*)px;  // x_s, run backwards from x_K
    double* VH = (double*)pv; // v_{s+1/2}
    vp.uni = (int*)pu;
    count(1);
    NB_CUDA(nbk::uniform_mass_flag(n, mass, vp.uni, st));
    NB_CUDA(cudaMemcpyAsync(X, xK, n3b, cudaMemcpyDeviceToDevice, st));
    NB_CUDA(cudaMemcpyAsync(VH, vK, n3b, cudaMemcpyDeviceToDevice, st));

    // The sweep needs the positions x_s of every step, newest first.  It runs
    // the leapfrog backwards from (x_K, v_{K-1/2}):
    //   x_s = x_{s+1} - dt v_{s+1/2},   v_{s-1/2} = v_{s+1/2} - dt a(x_s),
    // with a(x_s) from the VJP kernel at x_s itself (its FORCE variant: the
    // same pair terms, 3 or 4 more FMAs per pair), and takes (x_c, v_{c+1/2})
    // from the tape at every checkpoint c, so a reversed state is never more
    // than ckpt_every - 1 steps from a recorded one.  No forward replay.
    // Every VJP but the last is consumed by the next pack_vjp, which adds the
    // split blocks' partial sums itself (and those of the force).
    nbk::SplitSums ss, ss_acc;
    // v_K = v_{K-1/2} + h a(x_K): the closing kick's VJP at x_K
    count(2);
    NB_CUDA(nbk::pack_vjp(n, vp.npad, vp.block, X, mass, nullptr, lamv, lamx, nullptr, nullptr, gm_acc, 0.0, h,
                          nullptr, plain, vp.jv, vp.centres, st));
    NB_CHECK(run_vjp(vp, n, eps2, !plain, false, g, gm, c.sms, st, &ss));
    bool have_a = false;  // a holds (or defers) the force at x_{s+1}
    for (int64_t s = steps - 1; s >= 0; --s) {
        nbk::ReverseStep rev;
        rev.x = X;
        rev.vh = VH;
        if (s % ckpt_every == 0) {  // a checkpoint: the recorded state
            const double* slot = tp + (size_t)(s / ckpt_every) * 2 * n * 3;
            rev.anchor_x = slot;
            rev.anchor_v = slot + (size_t)n * 3;
        } else {
            rev.a = have_a ? a : nullptr;  // s = steps - 1 starts from v_{K-1/2} itself
            rev.ss_acc = ss_acc;
            rev.kick = have_a ? dt : 0.0;
            rev.drift = dt;
        }
        const double kappa = (s == 0) ? h : dt;
        const int64_t it = steps - 1 - s;
        if (plain) {
            count(2);
            NB_CUDA(nbk::pack_vjp(n, vp.npad, vp.block, X, mass, nullptr, lamv, lamx, g, gm, gm_acc, dt, kappa,
                                  nullptr, plain, vp.jv, vp.centres, st, &ss, &rev));
        } else {  // one kernel: cell centres from the previous step's chunk sums
            count(1);
            NB_CUDA(nbk::pack_vjp_lagged(n, vp.npad, vp.block, mass, lamv, lamx, g, gm, gm_acc, dt, kappa, vp.jv,
                                         vp.centres, vp.chunks[it & 1], vp.chunks[(it + 1) & 1], st, &ss, &rev));
        }
        // the force at x_s is needed to step back to x_{s-1} unless that is a checkpoint
        const bool want_a = s > 0 && (s - 1) % ckpt_every != 0;
        NB_CHECK(run_vjp(vp, n, eps2, !plain, false, g, gm, c.sms, st, s > 0 ? &ss : nullptr, want_a ? a : nullptr,
                         want_a ? &ss_acc : nullptr));
        have_a = want_a;
    }
    count(1);
    NB_CUDA(nbk::adjoint_accumulate(n, lamx, g, gm_acc, gm, st));
    return sg.finish();
}

// The adjoint in one call from x(0), v(0): the forward run is recorded into
// workspace copies of the state and a workspace tape, then swept.  Buffers of
// its own (B_VJ*) hold those, so the staging inside the two calls it makes
// cannot overwrite them.
int nbody_leapfrog_vjp(int64_t n, const double* pos0, const double* vel0, const float* mass, double eps, double dt,
                       int64_t steps, int64_t ckpt_every, const double* g_posT, const double* g_velT, double* g_pos0,
                       double* g_vel0, double* g_mass, const nbody_opts* opts) {
    NB_RANGE("nbody_leapfrog_vjp");
    if (n < 0 || steps < 0 || ckpt_every < 1 || !finite_nonneg(eps) || !isfinite(dt)) return NBODY_EINVAL;
    if (n > 0 && (pos0 == nullptr || vel0 == nullptr || mass == nullptr || g_posT == nullptr || g_velT == nullptr ||
                  g_pos0 == nullptr || g_vel0 == nullptr || g_mass == nullptr))
        return NBODY_EINVAL;
    NB_CHECK(check_opts_only(opts));
    if (n == 0) return NBODY_OK;
    Ctx c;
    NB_CHECK(begin(opts, &c));
    cudaStream_t st = c.o.stream;
    const size_t n3b = (size_t)n * 3 * sizeof(double);
    const int64_t tb = nbody_tape_bytes(n, steps, ckpt_every);
    void *px, *pv, *pm, *pt;
    NB_CHECK(ensure(c.ws, B_VJX, n3b, &px));
    NB_CHECK(ensure(c.ws, B_VJV, n3b, &pv));
    NB_CHECK(ensure(c.ws, B_VJM, (size_t)n * sizeof(float), &pm));
    NB_CHECK(ensure(c.ws, B_VJTAPE, (size_t)tb, &pt));
    // cudaMemcpyDefault: the sources may be host (pageable or pinned) or device memory
    NB_CUDA(cudaMemcpyAsync(px, pos0, n3b, cudaMemcpyDefault, st));
    NB_CUDA(cudaMemcpyAsync(pv, vel0, n3b, cudaMemcpyDefault, st));
    NB_CUDA(cudaMemcpyAsync(pm, mass, (size_t)n * sizeof(float), cudaMemcpyDefault, st));
    NB_CHECK(nbody_leapfrog_record(n, (double*)px, (double*)pv, (const float*)pm, eps, dt, steps, ckpt_every, pt,
                                   opts));
    return nbody_leapfrog_vjp_tape(n, (const float*)pm, eps, dt, steps, ckpt_every, pt, g_posT, g_velT, g_pos0,
                                   g_vel0, g_mass, opts);
}

// Ragged batches.  With the offsets in host memory the batch is checked on
// the host (errors return before any work is queued) and its largest system
// picks the kernel shape; with device offsets the checks run on the device
// (a bad batch is skipped and nbody_last_device_error reports NBODY_EINVAL)
// and shape 0 serves unless opts->config names another.  The order of the
// systems and the split of the large ones are planned on the device in
// either case, so a call on device arrays never waits for the GPU.
static int batched_common(int64_t nsys, const int64_t* offsets, float* pos, float* vel, const float* mass,
                          const float* eps, float* acc, float* pot, double dt, int64_t steps, const nbody_opts* opts,
                          bool leapfrog) {
    if (nsys < 0 || steps < 0 || !isfinite(dt)) return NBODY_EINVAL;
    if (nsys > 0 && (offsets == nullptr || pos == nullptr || mass == nullptr || eps == nullptr)) return NBODY_EINVAL;
    if (nsys > 0 && leapfrog && vel == nullptr) return NBODY_EINVAL;
    if (nsys > 0 && !leapfrog && acc == nullptr) return NBODY_EINVAL;
    NB_CHECK(check_opts_only(opts, nbk::batched_num_shapes()));
    if (nsys == 0 || (leapfrog && steps == 0)) return NBODY_OK;
    if (nsys > (int64_t)1 << 30) return NBODY_EINVAL;
    Ctx c;
    NB_CHECK(begin(opts, &c, nbk::batched_num_shapes()));
    cudaStream_t st = c.o.stream;
    int64_t max_ns = -1, ntot = -1;  // -1: not known on the host
    if (is_host_ptr(offsets)) {
        if (offsets[0] != 0) return NBODY_EINVAL;
        max_ns = 0;
        for (int64_t s = 0; s < nsys; ++s) {
            const int64_t ns = offsets[s + 1] - offsets[s];
            if (ns < 0 || ns > INT32_MAX) return NBODY_EINVAL;
            max_ns = ns > max_ns ? ns : max_ns;
        }
        ntot = offsets[nsys];
        if (is_host_ptr(eps))
            for (int64_t s = 0; s < nsys; ++s)
                if (!(isfinite(eps[s]) && eps[s] >= 0.0f)) return NBODY_EINVAL;
        if (ntot == 0) return NBODY_OK;
    }
    const bool host_data = is_host_ptr(pos) || (leapfrog && is_host_ptr(vel)) || is_host_ptr(mass) ||
                           (!leapfrog && is_host_ptr(acc)) || (!leapfrog && pot != nullptr && is_host_ptr(pot));
    if (host_data && ntot < 0) {
        // host arrays are copied in and out, so their size must be known: read
        // the batch's body count back (the call is synchronous anyway)
        NB_CUDA(cudaMemcpyAsync(&ntot, offsets + nsys, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        NB_CUDA(cudaStreamSynchronize(st));
        if (ntot < 0) return NBODY_EINVAL;
        if (ntot == 0) return NBODY_OK;
    }
    const size_t nb = ntot > 0 ? (size_t)ntot : 0;
    Staging sg(c.ws);
    sg.add(offsets, (size_t)(nsys + 1) * sizeof(int64_t), true, false);
    sg.add(pos, nb * 3 * sizeof(float), true, leapfrog);
    sg.add(vel, leapfrog ? nb * 3 * sizeof(float) : 0, leapfrog, leapfrog);
    sg.add(mass, nb * sizeof(float), true, false);
    sg.add(eps, (size_t)nsys * sizeof(float), true, false);
    sg.add(acc, leapfrog ? 0 : nb * 3 * sizeof(float), false, !leapfrog);
    sg.add(pot, (leapfrog || pot == nullptr) ? 0 : nb * sizeof(float), false, !leapfrog);
    NB_CHECK(sg.prepare());
    const int shape = c.o.config >= 0 ? c.o.config : (max_ns >= 0 ? tuned_shape(2, max_ns, 0) : 0);
    const int maxcap = nbk::batched_max_cap(shape);
    nbk::BatchArgs a;
    if (max_ns >= 0 && max_ns <= maxcap) {  // every system fits one CTA's image
        a.cap = max_ns > 2 ? (int)max_ns : 2;
        a.coop = false;
    } else {  // sizes unknown here, or some system too large for one image
        a.cap = maxcap;
        a.coop = true;
    }
    void *pb, *pe;
    NB_CHECK(ensure(c.ws, B_BATCH, nbk::batched_scratch_bytes(nsys), &pb));
    NB_CHECK(ensure(c.ws, B_ERR, sizeof(int), &pe));
    if (fault("launch")) return NBODY_ECUDA;
    a.nsys = nsys;
    a.offsets = (const int64_t*)sg.dev(0);
    a.pos = (float*)sg.dev(1);
    a.vel = leapfrog ? (float*)sg.dev(2) : nullptr;
    a.mass = (const float*)sg.dev(3);
    a.eps = (const float*)sg.dev(4);
    a.acc = leapfrog ? nullptr : (float*)sg.dev(5);
    a.pot = (leapfrog || pot == nullptr) ? nullptr : (float*)sg.dev(6);
    a.dt = (float)dt;
    a.steps = leapfrog ? steps : 0;
    a.scratch = pb;
    a.err = (int*)pe;
    const std::vector<uint64_t> key = {2, (uint64_t)nsys, (uint64_t)(uintptr_t)a.offsets,
                                       (uint64_t)(uintptr_t)a.pos, (uint64_t)(uintptr_t)a.vel,
                                       (uint64_t)(uintptr_t)a.mass, (uint64_t)(uintptr_t)a.eps,
                                       (uint64_t)(uintptr_t)a.acc, (uint64_t)(uintptr_t)a.pot, bits_of(dt),
                                       (uint64_t)a.steps, (uint64_t)shape, (uint64_t)a.cap, (uint64_t)a.coop,
                                       (uint64_t)(uintptr_t)pb, (uint64_t)(uintptr_t)pe};
    NB_CHECK(run_graphed(c, key, true, [&](cudaStream_t s) {
        int launched = 0;
        const cudaError_t e = nbk::batched_launch(shape, a, c.sms, s, &launched);
        count(launched);
        NB_CUDA(e);
        return NBODY_OK;
    }));
    return sg.finish();
}

int nbody_accel_batched(int64_t nsys, const int64_t* offsets, const float* pos, const float* mass, const float* eps,
                        float* acc, float* pot, const nbody_opts* opts) {
    NB_RANGE("nbody_accel_batched");
    return batched_common(nsys, offsets, const_cast<float*>(pos), nullptr, mass, eps, acc, pot, 0.0, 0, opts, false);
}

int nbody_leapfrog_batched(int64_t nsys, const int64_t* offsets, float* pos, float* vel, const float* mass,
                           const float* eps, double dt, int64_t steps, const nbody_opts* opts) {
    NB_RANGE("nbody_leapfrog_batched");
    return batched_common(nsys, offsets, pos, vel, mass, eps, nullptr, nullptr, dt, steps, opts, true);
}

static int energy_common(int64_t n, const void* pos, const void* vel, const float* mass, double eps, double* out,
                         const nbody_opts* opts, bool f64) {
    if (n < 0 || !finite_nonneg(eps) || out == nullptr) return NBODY_EINVAL;
    if (n > 0 && (pos == nullptr || vel == nullptr || mass == nullptr)) return NBODY_EINVAL;
    NB_CHECK(check_opts_only(opts));
    if (n == 0) {
        for (int k = 0; k < 9; ++k) out[k] = 0.0;
        return NBODY_OK;
    }
    Ctx c;
    NB_CHECK(begin(opts, &c));
    const size_t vb = f64 ? sizeof(double) : sizeof(float);
    Staging sg(c.ws);
    sg.add(pos, (size_t)n * 3 * vb, true, false);
    sg.add(vel, (size_t)n * 3 * vb, true, false);
    sg.add(mass, (size_t)n * sizeof(float), true, false);
    NB_CHECK(sg.prepare());
    void *pa, *pp, *pr, *po;
    NB_CHECK(ensure(c.ws, B_ACC, (size_t)n * 3 * sizeof(float), &pa));
    NB_CHECK(ensure(c.ws, B_POT, (size_t)n * sizeof(float), &pp));
    NB_CHECK(ensure(c.ws, B_RED, nbk::reduce_scratch_doubles() * sizeof(double), &pr));
    NB_CHECK(ensure(c.ws, B_OUT9, 9 * sizeof(double), &po));
    if (f64) {
        NB_CHECK(accel_f64_dev(c, n, (const double*)sg.dev(0), (const float*)sg.dev(2), eps, (float*)pa, (float*)pp));
        count(2);
        NB_CUDA(nbk::energy_reduce_f64(n, (const double*)sg.dev(1), (const float*)sg.dev(2), (const float*)pa,
                                       (const float*)pp, (double*)pr, (double*)po, c.o.stream));
    } else {
        NB_CHECK(accel_f32_dev(c, n, (const float*)sg.dev(0), (const float*)sg.dev(2), (float)eps, (float*)pa,
                               (float*)pp));
        count(2);
        NB_CUDA(nbk::energy_reduce_f32(n, (const float*)sg.dev(1), (const float*)sg.dev(2), (const float*)pa,
                                       (const float*)pp, (double*)pr, (double*)po, c.o.stream));
    }
    NB_CUDA(cudaMemcpyAsync(out, po, 9 * sizeof(double), cudaMemcpyDeviceToHost, c.o.stream));
    NB_CUDA(cudaStreamSynchronize(c.o.stream));
    return sg.finish();
}

int nbody_energy(int64_t n, const double* pos, const double* vel, const float* mass, double eps, double* out,
                 const nbody_opts* opts) {
    NB_RANGE("nbody_energy");
    return energy_common(n, pos, vel, mass, eps, out, opts, true);
}

int nbody_energy_f32(int64_t n, const float* pos, const float* vel, const float* mass, float eps, double* out,
                     const nbody_opts* opts) {
    NB_RANGE("nbody_energy_f32");
    return energy_common(n, pos, vel, mass, (double)eps, out, opts, false);
}

int nbody_last_device_error(void) {
    int dev = 0;
    NB_CUDA(cudaGetDevice(&dev));
    NB_CUDA(cudaDeviceSynchronize());
    int result = NBODY_OK;
    std::lock_guard<std::mutex> lk(g_ws_mu);
    for (auto& kv : g_ws) {
        Workspace* w = kv.second;
        if (w->device != dev || w->buf[B_ERR].p == nullptr) continue;
        int flag = 0;
        NB_CUDA(cudaMemcpy(&flag, w->buf[B_ERR].p, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag != 0) {
            result = flag == nbk::kErrBounds ? NBODY_EBOUNDS
                     : flag == nbk::kErrInvalid ? NBODY_EINVAL
                                                : NBODY_ETIMEOUT;
            NB_CUDA(cudaMemset(w->buf[B_ERR].p, 0, sizeof(int)));
        }
    }
    return result;
}

int nbody_selftest_wait(double limit_seconds, const nbody_opts* opts) {
    NB_RANGE("nbody_selftest_wait");
    if (!(limit_seconds >= 1e-6 && limit_seconds <= 1.0)) return NBODY_EINVAL;
    NB_CHECK(check_opts_only(opts));
    Ctx c;
    NB_CHECK(begin(opts, &c));
    void* p;
    NB_CHECK(ensure(c.ws, B_ERR, sizeof(int), &p));
    count(1);
    NB_CUDA(nbk::selftest_wait((uint64_t)(limit_seconds * 1e9), (int*)p, c.o.stream));
    NB_CUDA(cudaStreamSynchronize(c.o.stream));
    int flag = 0;
    NB_CUDA(cudaMemcpy(&flag, p, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag != 0) {
        NB_CUDA(cudaMemset(p, 0, sizeof(int)));
        return NBODY_ETIMEOUT;
    }
    return NBODY_OK;
}

int nbody_tune_load(const char* path) {
    std::vector<TuneRule> r;
    const std::string p = path != nullptr ? std::string(path) : default_tune_path();
    int k = p.empty() ? NBODY_EINVAL : tune_parse(p.c_str(), r);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (k <= 0) {
        if (path == nullptr) {  // no file beside the library: the built-in table
            tune_defaults(g_tune);
            g_tune_loaded = true;
            return 0;
        }
        return NBODY_EINVAL;
    }
    g_tune = r;
    g_tune_loaded = true;
    return k;
}

int nbody_tuned_shape(int kind, int64_t n, int pot) {
    if (kind < 0 || kind > 2 || n < 0 || pot < 0 || pot > 1) return NBODY_EINVAL;
    return tuned_shape(kind, n, pot);
}

void nbody_profile_enable(int on) { g_prof_on.store(on != 0); }

int nbody_profile_read(double* force_ms, int64_t* force_launches, int64_t* all_launches) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    NB_CUDA(prof_drain());
    if (force_ms) *force_ms = g_prof_ms[PROF_FORCE];
    if (force_launches) *force_launches = g_prof_n[PROF_FORCE];
    g_prof_ms[PROF_FORCE] = 0.0;
    g_prof_n[PROF_FORCE] = 0;
    if (all_launches) *all_launches = g_launches.exchange(0);
    return NBODY_OK;
}

int nbody_profile_read_kind(int kind, double* ms, int64_t* launches) {
    if (kind < 0 || kind >= PROF_KINDS) return NBODY_EINVAL;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    NB_CUDA(prof_drain());
    if (ms) *ms = g_prof_ms[kind];
    if (launches) *launches = g_prof_n[kind];
    g_prof_ms[kind] = 0.0;
    g_prof_n[kind] = 0;
    return NBODY_OK;
}

void nbody_finalize(void) {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        (void)cudaGetLastError();
        cur = 0;
    }
    for (auto& kv : g_ws) {
        Workspace* w = kv.second;
        if (cudaSetDevice(w->device) == cudaSuccess) {
            (void)cudaDeviceSynchronize();
            for (int k = 0; k < NBUF; ++k)
                if (w->buf[k].p) (void)cudaFree(w->buf[k].p);
            if (w->aux != nullptr) {
                for (auto& e : w->ev) (void)cudaEventDestroy(e);
                (void)cudaStreamDestroy(w->aux);
            }
            for (auto& kv2 : w->graphs) drop_graph(kv2.second);
            if (w->cap != nullptr) (void)cudaStreamDestroy(w->cap);
        }
        delete w;
    }
    g_ws.clear();
    (void)cudaSetDevice(cur);
    (void)cudaGetLastError();
}

}  // extern "C"

// Programmatic dependent launch of the step kernels (nbody_internal.cuh):
// off while kernels are timed one by one, or when NBODY_NO_PDL is set.
bool nbk::pdl_on() {
    static const bool env_off = getenv("NBODY_NO_PDL") != nullptr;
    return !env_off && !g_prof_on.load();
}
