// tune.cu -- the process-wide table of tuned launch parameters (host code).
//
// Keys are (knob, N, M, precision, L class, SM count); the launchers of the
// contractions and of the persistent CG loop look their shape up here and
// fall back to their built-in heuristics when it has no entry.  The timing
// that fills the table (spirec_autotune) lives with the plan in capi.cu.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.cuh"

namespace spirec {
namespace {

using Key = std::tuple<int, int, int, int, int, int>;  // knob, N, M, precision, L class, sms

std::mutex g_mu;
std::map<Key, int>& table()
{
    static std::map<Key, int> t;
    return t;
}
std::atomic<unsigned> g_generation{1};

constexpr const char* kHeader = "spirec-tune 1";

bool valid_shape(int knob, int N, int M, int precision, int64_t L, int sms)
{
    if (knob < 0 || knob >= SPIREC_NUM_KNOBS) return false;
    if (precision != SPIREC_FP32 && precision != SPIREC_MIXED_FP16X3 && precision != SPIREC_MIXED_BF16X3)
        return false;
    if (N < 2 || M < 2 * N - 1 || L < 1 || sms < 0) return false;
    return true;
}

Key make_key(int knob, int N, int M, int precision, int64_t L, int sms)
{
    return Key{knob, N, M, precision, knob == SPIREC_KNOB_LOOP_ROWS ? 0 : l_class(L), sms};
}

int current_sms(int* sms)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("no CUDA device to take the SM count from (%s)", cudaGetErrorString(e));
        return SPIREC_ECUDA;
    }
    return SPIREC_OK;
}

// sms == 0 -> the current device's; validates the shape.
int resolve(int knob, int N, int M, int precision, int64_t L, int* sms)
{
    if (!valid_shape(knob, N, M, precision, L, *sms)) {
        set_error("bad tuning key (knob %d, N %d, M %d, precision %d, L %lld, sms %d)", knob, N, M, precision,
                  (long long)L, *sms);
        return SPIREC_EINVAL;
    }
    if (*sms == 0) return current_sms(sms);
    return SPIREC_OK;
}

}  // namespace

int l_class(int64_t L)
{
    int c = 0;
    while (c < 62 && ((int64_t)1 << c) < L) ++c;
    return c;
}

int tune_lookup(int knob, const spirec_plan_s* p, int sms)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto& t = table();
    if (t.empty()) return 0;
    auto it = t.find(make_key(knob, p->N, p->M, p->precision, p->L, sms));
    return it == t.end() ? 0 : it->second;
}

unsigned tune_generation() { return g_generation.load(); }

int device_sms(int* sms)
{
    int dev = 0;
    SPIREC_CK(cudaGetDevice(&dev));
    SPIREC_CK(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev));
    return SPIREC_OK;
}

int tune_store(int knob, const spirec_plan_s* p, int sms, int value)
{
    std::lock_guard<std::mutex> lk(g_mu);
    const Key k = make_key(knob, p->N, p->M, p->precision, p->L, sms);
    if (value > 0)
        table()[k] = value;
    else
        table().erase(k);
    g_generation.fetch_add(1);
    return SPIREC_OK;
}

}  // namespace spirec

using namespace spirec;

extern "C" {

int spirec_tune_set(int32_t knob, int32_t N, int32_t M, int32_t precision, int64_t L, int32_t sms, int32_t value)
{
    if (value < 0) {
        set_error("tuned value must be >= 0 (0 removes the entry)");
        return SPIREC_EINVAL;
    }
    int rc = resolve(knob, N, M, precision, L, &sms);
    if (rc != SPIREC_OK) return rc;
    std::lock_guard<std::mutex> lk(g_mu);
    const Key k = make_key(knob, N, M, precision, L, sms);
    if (value > 0)
        table()[k] = value;
    else
        table().erase(k);
    g_generation.fetch_add(1);
    return SPIREC_OK;
}

int spirec_tune_get(int32_t knob, int32_t N, int32_t M, int32_t precision, int64_t L, int32_t sms, int32_t* value)
{
    if (!value) {
        set_error("value must not be NULL");
        return SPIREC_EINVAL;
    }
    int rc = resolve(knob, N, M, precision, L, &sms);
    if (rc != SPIREC_OK) return rc;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = table().find(make_key(knob, N, M, precision, L, sms));
    *value = it == table().end() ? 0 : it->second;
    return SPIREC_OK;
}

int spirec_tune_count(int64_t* count)
{
    if (!count) {
        set_error("count must not be NULL");
        return SPIREC_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    *count = (int64_t)table().size();
    return SPIREC_OK;
}

int spirec_tune_clear(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    table().clear();
    g_generation.fetch_add(1);
    return SPIREC_OK;
}

int spirec_tune_save(const char* path)
{
    if (!path) {
        set_error("path must not be NULL");
        return SPIREC_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    FILE* fp = fopen(path, "w");
    if (!fp) {
        set_error("cannot open %s for writing", path);
        return SPIREC_EINVAL;
    }
    fprintf(fp, "%s\n", kHeader);
    for (const auto& kv : table()) {
        const Key& k = kv.first;
        fprintf(fp, "%d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k),
                std::get<4>(k), std::get<5>(k), kv.second);
    }
    const bool ok = fflush(fp) == 0;
    if (fclose(fp) != 0 || !ok) {
        set_error("write to %s failed", path);
        return SPIREC_EINVAL;
    }
    return SPIREC_OK;
}

// Lines: "knob N M precision lclass sms value".  The whole file is parsed
// before the table changes.
int spirec_tune_load(const char* path)
{
    if (!path) {
        set_error("path must not be NULL");
        return SPIREC_EINVAL;
    }
    FILE* fp = fopen(path, "r");
    if (!fp) {
        set_error("cannot open %s", path);
        return SPIREC_EINVAL;
    }
    char line[256];
    std::map<Key, int> add;
    int lineno = 0, rc = SPIREC_OK;
    while (fgets(line, sizeof line, fp)) {
        ++lineno;
        const size_t n = strlen(line);
        if (n == sizeof line - 1 && line[n - 1] != '\n') {
            set_error("%s:%d: line too long", path, lineno);
            rc = SPIREC_EINVAL;
            break;
        }
        if (lineno == 1) {
            if (strncmp(line, kHeader, strlen(kHeader)) != 0) {
                set_error("%s: not a tuning table (header \"%s\" missing)", path, kHeader);
                rc = SPIREC_EINVAL;
                break;
            }
            continue;
        }
        int v[7], used = 0;
        if (sscanf(line, "%d %d %d %d %d %d %d %n", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6], &used) != 7 ||
            line[used] != '\0') {
            set_error("%s:%d: malformed entry", path, lineno);
            rc = SPIREC_EINVAL;
            break;
        }
        const int64_t L = (int64_t)1 << (v[4] < 0 ? 0 : v[4] > 62 ? 62 : v[4]);
        if (!valid_shape(v[0], v[1], v[2], v[3], L, v[5]) || v[5] == 0 || v[4] < 0 || v[4] > 62 || v[6] <= 0 ||
            (v[0] == SPIREC_KNOB_LOOP_ROWS && v[4] != 0)) {
            set_error("%s:%d: entry out of range", path, lineno);
            rc = SPIREC_EINVAL;
            break;
        }
        add[Key{v[0], v[1], v[2], v[3], v[4], v[5]}] = v[6];
    }
    if (rc == SPIREC_OK && lineno == 0) {
        set_error("%s: empty file", path);
        rc = SPIREC_EINVAL;
    }
    fclose(fp);
    if (rc != SPIREC_OK) return rc;
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto& kv : add) table()[kv.first] = kv.second;
    g_generation.fetch_add(1);
    return SPIREC_OK;
}

}  // extern "C"
