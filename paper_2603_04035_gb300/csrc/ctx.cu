// Context management, error plumbing, device-wide scan and the host a,b fit.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>

#include "common.cuh"

namespace drgb {

int set_error(Ctx* c, int code, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

int ensure_scratch(Ctx* c, size_t bytes, cudaStream_t stream) {
    if (bytes <= c->scratch_bytes) return DRGB_OK;
    if (c->scratch_limit && bytes > c->scratch_limit)
        return set_error(c, DRGB_ERR_WORKSPACE, "scratch of %zu bytes needed, above the context's limit of %zu bytes",
                         bytes, c->scratch_limit);
    if (c->scratch) {
        DRGB_CUDA(c, cudaStreamSynchronize(stream));
        DRGB_CUDA(c, cudaFree(c->scratch));
        c->scratch = nullptr;
        c->scratch_bytes = 0;
    }
    size_t want = bytes + bytes / 8;  // headroom against frequent regrowth
    if (c->scratch_limit && want > c->scratch_limit) want = c->scratch_limit;
    cudaError_t e = cudaMalloc(&c->scratch, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(c, DRGB_ERR_CUDA, "scratch allocation of %zu bytes failed: %s", want,
                         cudaGetErrorString(e));
    }
    c->scratch_bytes = want;
    return DRGB_OK;
}

int stage_mark(Ctx* c, int idx, cudaStream_t st) {
    if (!c->profiling || idx < 0 || idx >= 11) return DRGB_OK;
    if (!c->stage_ev[idx]) DRGB_CUDA(c, cudaEventCreate(&c->stage_ev[idx]));
    DRGB_CUDA(c, cudaEventRecord(c->stage_ev[idx], st));
    if (idx < 6 && idx + 1 > c->stage_marks) c->stage_marks = idx + 1;
    if (idx >= 6) c->knn_marks |= 1u << (idx - 6);
    return DRGB_OK;
}

// ------------------------------------------------------------------ scan
static constexpr int SCAN_THREADS = 256;
static constexpr int SCAN_PER_THREAD = 8;
static constexpr int SCAN_BLOCK = SCAN_THREADS * SCAN_PER_THREAD;

__global__ void __launch_bounds__(SCAN_THREADS)
scan_block_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n,
                  int32_t* __restrict__ block_sums) {
    __shared__ int32_t warp_tot[SCAN_THREADS / 32];
    const int64_t base = int64_t(blockIdx.x) * SCAN_BLOCK + int64_t(threadIdx.x) * SCAN_PER_THREAD;
    int32_t v[SCAN_PER_THREAD];
    int32_t s = 0;
#pragma unroll
    for (int t = 0; t < SCAN_PER_THREAD; ++t) {
        v[t] = (base + t < n) ? in[base + t] : 0;
        s += v[t];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int32_t wt = lane < SCAN_THREADS / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, wt, o);
            if (lane >= o) wt += y;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = wt;  // inclusive over warps
    }
    __syncthreads();
    int32_t run = incl - s + (wid ? warp_tot[wid - 1] : 0);
#pragma unroll
    for (int t = 0; t < SCAN_PER_THREAD; ++t) {
        if (base + t < n) out[base + t] = run;
        run += v[t];
    }
    if (threadIdx.x == SCAN_THREADS - 1 && block_sums) block_sums[blockIdx.x] = run;
}

__global__ void scan_add_kernel(int32_t* __restrict__ out, int64_t n,
                                const int32_t* __restrict__ offs) {
    const int64_t i = int64_t(blockIdx.x) * SCAN_BLOCK + threadIdx.x;
#pragma unroll
    for (int t = 0; t < SCAN_PER_THREAD; ++t) {
        int64_t j = i + int64_t(t) * SCAN_THREADS;
        if (j < n) out[j] += offs[blockIdx.x];
    }
}

size_t scan_scratch_elems(int64_t n) {
    size_t total = 0;
    int64_t m = n;
    while (m > 0) {
        int64_t nb = (m + SCAN_BLOCK - 1) / SCAN_BLOCK;
        total += size_t(nb) * 2 + 2;
        if (nb <= 1) break;
        m = nb;
    }
    return total + 2;
}

// out[0..n] = exclusive scan of in[0..n), out[n] = total.
static int scan_rec(Ctx* c, const int32_t* in, int32_t* out, int64_t n, int32_t* tmp,
                    cudaStream_t st) {
    const int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    int32_t* sums = tmp;           // nb block totals
    int32_t* sums_scan = tmp + nb; // nb + 1 scanned totals
    scan_block_kernel<<<unsigned(nb), SCAN_THREADS, 0, st>>>(in, out, n, sums);
    DRGB_CHECK_LAUNCH(c);
    if (nb == 1) {
        // total = block sum; copy into out[n]
        DRGB_CUDA(c, cudaMemcpyAsync(out + n, sums, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        return DRGB_OK;
    }
    int rc = scan_rec(c, sums, sums_scan, nb, tmp + 2 * nb + 2, st);
    if (rc) return rc;
    scan_add_kernel<<<unsigned(nb), SCAN_THREADS, 0, st>>>(out, n, sums_scan);
    DRGB_CHECK_LAUNCH(c);
    DRGB_CUDA(c, cudaMemcpyAsync(out + n, sums_scan + nb, sizeof(int32_t),
                                 cudaMemcpyDeviceToDevice, st));
    return DRGB_OK;
}

int exclusive_scan(Ctx* c, const int32_t* in, int32_t* out, int64_t n, int32_t* tmp,
                   cudaStream_t st) {
    if (n <= 0) {
        DRGB_CUDA(c, cudaMemsetAsync(out, 0, sizeof(int32_t), st));
        return DRGB_OK;
    }
    return scan_rec(c, in, out, n, tmp, st);
}

// ------------------------------------------------------------------ tuning cache
// The file is a JSON object with one entry per line, written by this library:
//   {
//     "<key>": {"epoch_warps": 8, "epoch_pipe": 1},
//     ...
//   }
// Keys are printable ASCII without quotes or backslashes.  Reading accepts
// exactly the lines of that form and ignores every other line.

// A tuned epoch setting: force-kernel width and form.
struct TunedEpoch {
    int warps;
    int pipe;
};

bool cache_key_ok(const char* k) {
    if (!k || !*k) return false;
    size_t n = 0;
    for (const char* p = k; *p; ++p, ++n) {
        const unsigned char ch = static_cast<unsigned char>(*p);
        if (ch < 0x20 || ch > 0x7e || ch == '"' || ch == '\\') return false;
    }
    return n < 256;
}

std::map<std::string, TunedEpoch> cache_read(const char* path) {
    std::map<std::string, TunedEpoch> m;
    FILE* f = std::fopen(path, "r");
    if (!f) return m;
    char line[1024];
    while (std::fgets(line, sizeof(line), f)) {
        const char* p = std::strchr(line, '"');
        if (!p) continue;
        const char* q = std::strchr(p + 1, '"');
        if (!q) continue;
        const std::string key(p + 1, q);
        const char* v = std::strstr(q + 1, "\"epoch_warps\":");
        if (!v || !cache_key_ok(key.c_str())) continue;
        char* end = nullptr;
        const long w = std::strtol(v + std::strlen("\"epoch_warps\":"), &end, 10);
        if (end == v || w < 1 || w > 1024) continue;
        long pp = 1;  // entries written before the form was tuned: the default form
        if (const char* u = std::strstr(q + 1, "\"epoch_pipe\":")) {
            char* e2 = nullptr;
            pp = std::strtol(u + std::strlen("\"epoch_pipe\":"), &e2, 10);
            if (e2 == u || pp < 0 || pp > 1) continue;
        }
        m[key] = TunedEpoch{int(w), int(pp)};
    }
    std::fclose(f);
    return m;
}

bool cache_write(const char* path, const std::map<std::string, TunedEpoch>& m) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return false;
    bool ok = std::fputs("{\n", f) >= 0;
    size_t i = 0;
    for (const auto& kv : m) {
        ok = ok && std::fprintf(f, "  \"%s\": {\"epoch_warps\": %d, \"epoch_pipe\": %d}%s\n", kv.first.c_str(),
                                kv.second.warps, kv.second.pipe, ++i < m.size() ? "," : "") > 0;
    }
    ok = ok && std::fputs("}\n", f) >= 0;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return false;
    }
    return true;
}

std::string tuning_key(const Ctx* c, int64_t rows, int64_t instances, int k) {
    auto lg = [](int64_t v) {
        int e = 0;
        while (v > 1) {
            v >>= 1;
            ++e;
        }
        return e;
    };
    char buf[384];
    std::snprintf(buf, sizeof(buf), "%s|%d SMs|rows 2^%d|instances 2^%d|k %d", c->device_name.c_str(), c->num_sms,
                  lg(rows), lg(instances), k);
    std::string s = buf;
    for (char& ch : s)
        if (ch == '"' || ch == '\\' || static_cast<unsigned char>(ch) < 0x20 || static_cast<unsigned char>(ch) > 0x7e)
            ch = '_';
    return s;
}


}  // namespace drgb

using namespace drgb;

extern "C" {

int drgb_version(void) { return 10000; }

int drgb_ctx_create(int device, drgb_ctx** out) {
    if (!out) return DRGB_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return DRGB_ERR_DEVICE;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return DRGB_ERR_CUDA;
    if (!(prop.major == 10 && prop.minor == 3)) return DRGB_ERR_DEVICE;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return DRGB_ERR_CUDA;
    drgb_ctx* c = new drgb_ctx();
    c->device = device;
    c->num_sms = prop.multiProcessorCount;
    c->l2_bytes = size_t(prop.l2CacheSize);
    c->smem_per_sm = size_t(prop.sharedMemPerMultiprocessor);
    c->device_name = prop.name;
    if (cudaMalloc(&c->d_status, 256) != cudaSuccess) {
        delete c;
        cudaSetDevice(prev);
        return DRGB_ERR_CUDA;
    }
    cudaMemset(c->d_status, 0, 256);
    c->d_counter = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(c->d_status) + 128);
    cudaDeviceSynchronize();
    cudaSetDevice(prev);
    *out = c;
    return DRGB_OK;
}

int drgb_ctx_destroy(drgb_ctx* c) {
    if (!c) return DRGB_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    if (c->epoch_exec) cudaGraphExecDestroy(c->epoch_exec);
    if (c->scratch) cudaFree(c->scratch);
    if (c->d_status) cudaFree(c->d_status);
    for (auto& e : c->stage_ev)
        if (e) cudaEventDestroy(e);
    cudaSetDevice(prev);
    delete c;
    return DRGB_OK;
}

const char* drgb_last_error(const drgb_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t drgb_ctx_scratch_bytes(const drgb_ctx* c) { return c ? int64_t(c->scratch_bytes) : 0; }

int drgb_set_scratch_limit(drgb_ctx* c, int64_t bytes) {
    if (!c) return DRGB_ERR_INVALID;
    if (bytes < 0) return set_error(c, DRGB_ERR_INVALID, "scratch limit must be >= 0");
    c->scratch_limit = size_t(bytes);
    if (bytes && c->scratch && c->scratch_bytes > size_t(bytes)) {  // honour the cap now
        DRGB_CUDA(c, cudaFree(c->scratch));  // waits for work that may still use it
        c->scratch = nullptr;
        c->scratch_bytes = 0;
    }
    return DRGB_OK;
}

int64_t drgb_launch_count(const drgb_ctx* c) { return c ? c->launches : 0; }

int drgb_set_tuning(drgb_ctx* c, int32_t param, int32_t value) {
    if (!c) return DRGB_ERR_INVALID;
    switch (param) {
        case DRGB_TUNE_EPOCH_WARPS:
            if (value != 4 && value != 8)
                return set_error(c, DRGB_ERR_INVALID, "epoch force-kernel width must be 4 or 8 warps");
            c->epoch_warps = value;
            return DRGB_OK;
        case DRGB_TUNE_EPOCH_PIPE:
            if (value != 0 && value != 1)
                return set_error(c, DRGB_ERR_INVALID, "epoch kernel form must be 0 (flat) or 1 (pipelined)");
            c->epoch_pipe = value;
            return DRGB_OK;
        default:
            return set_error(c, DRGB_ERR_INVALID, "unknown tuning parameter %d", param);
    }
}

int drgb_tuning_cache_lookup(const char* path, const char* key, int32_t* epoch_warps, int32_t* epoch_pipe) {
    if (!path || !*path || !drgb::cache_key_ok(key) || !epoch_warps || !epoch_pipe) return DRGB_ERR_INVALID;
    const auto m = drgb::cache_read(path);
    const auto it = m.find(key);
    if (it == m.end() || !drgb::epoch_warps_supported(it->second.warps)) return DRGB_ERR_INVALID;
    *epoch_warps = it->second.warps;
    *epoch_pipe = it->second.pipe;
    return DRGB_OK;
}

int drgb_tuning_cache_store(const char* path, const char* key, int32_t epoch_warps, int32_t epoch_pipe) {
    if (!path || !*path || !drgb::cache_key_ok(key) || !drgb::epoch_warps_supported(epoch_warps) ||
        (epoch_pipe != 0 && epoch_pipe != 1))
        return DRGB_ERR_INVALID;
    auto m = drgb::cache_read(path);
    m[key] = drgb::TunedEpoch{epoch_warps, epoch_pipe};
    return drgb::cache_write(path, m) ? DRGB_OK : DRGB_ERR_INVALID;
}

int drgb_set_tuning_cache(drgb_ctx* c, const char* path) {
    if (!c) return DRGB_ERR_INVALID;
    c->tuning_cache = path ? path : "";
    return DRGB_OK;
}

int drgb_get_tuning(const drgb_ctx* c, int32_t param, int32_t* value) {
    if (!c || !value) return DRGB_ERR_INVALID;
    switch (param) {
        case DRGB_TUNE_EPOCH_WARPS: *value = c->epoch_warps; return DRGB_OK;
        case DRGB_TUNE_EPOCH_PIPE: *value = c->epoch_pipe; return DRGB_OK;
        default: return DRGB_ERR_INVALID;
    }
}

int drgb_set_profiling(drgb_ctx* c, int on) {
    if (!c) return DRGB_ERR_INVALID;
    c->profiling = on != 0;
    c->stage_marks = 0;
    c->knn_marks = 0;
    return DRGB_OK;
}

int drgb_stage_times(drgb_ctx* c, float* ms, int max) {
    if (!c || !ms || max < 0) return DRGB_ERR_INVALID;
    int m = 0;
    for (int s = 0; s + 1 < c->stage_marks && m < max && s < 4; ++s, ++m) {
        DRGB_CUDA(c, cudaEventSynchronize(c->stage_ev[s + 1]));
        DRGB_CUDA(c, cudaEventElapsedTime(&ms[m], c->stage_ev[s], c->stage_ev[s + 1]));
    }
    auto span = [&](int a, int b, float* out) -> int {
        *out = 0.f;
        if ((c->knn_marks >> (a - 6) & 1u) && (c->knn_marks >> (b - 6) & 1u)) {
            DRGB_CUDA(c, cudaEventSynchronize(c->stage_ev[b]));
            DRGB_CUDA(c, cudaEventElapsedTime(out, c->stage_ev[a], c->stage_ev[b]));
        }
        return DRGB_OK;
    };
    // [4] the tensor-core k-NN kernel alone, [5] its ordering and staging,
    // [6] the re-rank, [7] the re-scan of uncertified rows (0 where the
    // tensor-core path did not run or, for [7], deferred its re-scan)
    static const int from[4] = {6, 8, 7, 9}, to[4] = {7, 6, 9, 10};
    for (int s = 0; m == 4 + s && m < max && s < 4; ++s, ++m) {
        int rc = span(from[s], to[s], &ms[m]);
        if (rc) return rc;
    }
    return m;
}

int drgb_sync(drgb_ctx* c, void* stream) {
    if (!c) return DRGB_ERR_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DRGB_CUDA(c, cudaStreamSynchronize(st));
    int status = 0;
    DRGB_CUDA(c, cudaMemcpy(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) {
        DRGB_CUDA(c, cudaMemset(c->d_status, 0, sizeof(int)));
        return set_error(c, status, "device-side error %d reported by a kernel", status);
    }
    return DRGB_OK;
}

int drgb_default_params(drgb_params* p) {
    if (!p) return DRGB_ERR_INVALID;
    std::memset(p, 0, sizeof(*p));
    p->k = 15;
    p->n_epochs = 200;
    p->neg = 5;
    p->lr0 = 1.0f;
    p->min_dist = 0.1f;
    p->spread = 1.0f;
    p->init_range = 10.0f;
    p->seed_init = 1;
    p->seed_neg = 2;
    p->knn_mode = 0;
    return DRGB_OK;
}

// Gauss-Newton least squares for Phi(x) = 1 / (1 + a x^(2b)) against the UMAP
// target curve on 300 points of [0, 3 spread]; each step is halved until the
// squared residual decreases.
int drgb_find_ab(float spread, float min_dist, float* a_out, float* b_out) {
    if (!a_out || !b_out || !(spread > 0.f) || !(min_dist >= 0.f)) return DRGB_ERR_INVALID;
    const int G = 300;
    double xs[G], ys[G], lx[G];
    for (int t = 0; t < G; ++t) {
        xs[t] = 3.0 * spread * t / (G - 1);
        ys[t] = xs[t] < min_dist ? 1.0 : std::exp(-(xs[t] - min_dist) / spread);
        lx[t] = xs[t] > 0 ? std::log(xs[t]) : 0.0;
    }
    auto cost = [&](double a, double b) {
        double s = 0;
        for (int t = 0; t < G; ++t) {
            double p = xs[t] > 0 ? std::exp(2.0 * b * lx[t]) : 0.0;
            double r = 1.0 / (1.0 + a * p) - ys[t];
            s += r * r;
        }
        return s;
    };
    double a = 1.0, b = 1.0, f = cost(a, b);
    for (int it = 0; it < 200; ++it) {
        double JtJ00 = 0, JtJ01 = 0, JtJ11 = 0, g0 = 0, g1 = 0;
        for (int t = 0; t < G; ++t) {
            if (!(xs[t] > 0)) {
                double r = 1.0 - ys[t];
                (void)r;  // derivative is zero at x = 0
                continue;
            }
            double p = std::exp(2.0 * b * lx[t]);
            double den = 1.0 + a * p;
            double r = 1.0 / den - ys[t];
            double ja = -p / (den * den);
            double jb = -a * p * 2.0 * lx[t] / (den * den);
            JtJ00 += ja * ja;
            JtJ01 += ja * jb;
            JtJ11 += jb * jb;
            g0 += ja * r;
            g1 += jb * r;
        }
        double det = JtJ00 * JtJ11 - JtJ01 * JtJ01;
        if (!(std::fabs(det) > 0)) break;
        double da = -(JtJ11 * g0 - JtJ01 * g1) / det;
        double db = -(-JtJ01 * g0 + JtJ00 * g1) / det;
        double lam = 1.0, fn = f, an = a, bn = b;
        bool moved = false;
        while (lam > 1e-12) {
            an = a + lam * da;
            bn = b + lam * db;
            if (an > 0 && bn > 0) {
                fn = cost(an, bn);
                if (fn < f) {
                    moved = true;
                    break;
                }
            }
            lam *= 0.5;
        }
        if (!moved) break;
        bool done = (f - fn) <= 1e-14 * (f > 1e-300 ? f : 1e-300);
        a = an;
        b = bn;
        f = fn;
        if (done) break;
    }
    *a_out = float(a);
    *b_out = float(b);
    return DRGB_OK;
}

}  // extern "C"
