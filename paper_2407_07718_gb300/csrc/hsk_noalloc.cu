// hsk_noalloc.cu -- the LSD key sort of stage S4 with no device allocation.
//
// Some callers cannot call cudaMalloc: a process whose device memory is all
// reserved up front by another allocator (a framework's caching allocator, a
// fixed arena), or code that must not take the device-wide synchronization
// that cudaMalloc/cudaFree can imply.  For them hsk_sort_keys_noalloc sorts
// keys the caller already holds, with its scratch -- the alternate key buffer,
// the look-back status words, the digit histograms and offsets -- in one
// file-scope __device__ array of fixed size that every GPU loading this
// library holds until the process exits.
//
// The array's name in host code is only a host-side stand-in, never a device
// address: the first call on each device (with that device current) asks the
// runtime for the array's device address with cudaGetSymbolAddress and keeps
// it for the life of the process.  A cudaDeviceReset reloads the module, after
// which that kept address is stale: do not call this entry point again after
// resetting the device.  All calls share the array and it keeps the last
// call's contents, so each call clears what must start at zero (histograms,
// status words, tile counters, error word).  Two calls that overlap on the GPU
// (different streams or host threads) race on the array.  Every call ends by
// reading the error word back and synchronizing its stream, so it is
// synchronous and cannot be recorded into a CUDA graph by stream capture.
#include <mutex>

#include "../../include/hsk_stages.h"
#include "hsk_internal.h"

namespace {

constexpr size_t ALT_BYTES = 8u << 20;                 // 2^20 x 8 B keys or 2^19 x 16 B keys
constexpr size_t STATUS_WORDS = 512 * 256;             // 512 tiles (of >= 2048 keys) x 256 digits
constexpr size_t HIST_WORDS = 16 * 256;                // up to 16 passes x 256 digits
constexpr size_t OFF_ALT = 0;
constexpr size_t OFF_STATUS = OFF_ALT + ALT_BYTES;
constexpr size_t OFF_HIST = OFF_STATUS + STATUS_WORDS * 8;
constexpr size_t OFF_DOFF = OFF_HIST + HIST_WORDS * 8;
constexpr size_t OFF_KEYBASE = OFF_DOFF + HIST_WORDS * 8;   // 2 words: {0, n}
constexpr size_t OFF_CTR = OFF_KEYBASE + 16;                 // 16 tile counters
constexpr size_t OFF_ERR = OFF_CTR + 16 * 4;                 // error word
constexpr size_t SCRATCH_BYTES = OFF_ERR + 256;

static_assert(HSK_NOALLOC_MAX_KEYS_U64 * 8 <= ALT_BYTES, "alternate buffer too small");
static_assert(HSK_NOALLOC_MAX_KEYS_U128 * 16 <= ALT_BYTES, "alternate buffer too small");

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch_addr[MAX_DEVICES] = {};
int g_num_sms[MAX_DEVICES] = {};

}  // namespace

static __device__ __align__(256) unsigned char g_sort_scratch[SCRATCH_BYTES];

__global__ void k_noalloc_key_base(unsigned long long* key_base, unsigned long long n) {
    if (threadIdx.x == 0) {
        key_base[0] = 0;
        key_base[1] = n;
    }
}

extern "C" int hsk_sort_keys_noalloc(uint64_t* d_keys, uint64_t n, int key_words, int key_bits, void* stream) {
    if ((key_words != 1 && key_words != 2) || key_bits < 1 || key_bits > 64 * key_words || (n && !d_keys))
        return HSK_EINVAL;
    // keys are read as whole words: 8-byte aligned, 128-bit keys 16-byte aligned
    if (reinterpret_cast<uintptr_t>(d_keys) % (8u * (unsigned)key_words)) return HSK_EINVAL;
    const uint64_t max_n = key_words == 1 ? HSK_NOALLOC_MAX_KEYS_U64 : HSK_NOALLOC_MAX_KEYS_U128;
    if (n > max_n) return HSK_EOVERFLOW;  // beyond the fixed scratch array
    if (n <= 1) return HSK_OK;
    // a launch error left pending by the caller's earlier work is neither
    // cleared nor taken for this call's own: the call does nothing
    if (cudaPeekAtLastError() != cudaSuccess) return HSK_ECUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return HSK_ECUDA;
    unsigned char* base = nullptr;
    int num_sms = 0;
    {
        std::lock_guard<std::mutex> g(g_mu);
        if (!g_scratch_addr[dev]) {  // set-up: once per device, with that device current
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess) return HSK_ECUDA;
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HSK_ECUDA;
            g_num_sms[dev] = sms;
            g_scratch_addr[dev] = p;
        }
        base = static_cast<unsigned char*>(g_scratch_addr[dev]);
        num_sms = g_num_sms[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int P = (key_bits + 7) / 8;
    const uint64_t tile_keys = hsk::onesweep_tile_keys(key_words);
    const uint64_t tiles = (n + tile_keys - 1) / tile_keys;
    if (tiles * 256 > STATUS_WORDS) return HSK_EOVERFLOW;
    void* alt = base + OFF_ALT;
    uint64_t* status = reinterpret_cast<uint64_t*>(base + OFF_STATUS);
    uint64_t* hist = reinterpret_cast<uint64_t*>(base + OFF_HIST);
    uint64_t* doff = reinterpret_cast<uint64_t*>(base + OFF_DOFF);
    uint64_t* key_base = reinterpret_cast<uint64_t*>(base + OFF_KEYBASE);
    uint32_t* ctr = reinterpret_cast<uint32_t*>(base + OFF_CTR);
    int* err = reinterpret_cast<int*>(base + OFF_ERR);
    // the array keeps the last call's contents: clear what must start at zero
    if (cudaMemsetAsync(hist, 0, (size_t)P * 256 * 8, st) != cudaSuccess) return HSK_ECUDA;
    if (cudaMemsetAsync(status, 0, (size_t)tiles * 256 * 8, st) != cudaSuccess) return HSK_ECUDA;
    if (cudaMemsetAsync(ctr, 0, OFF_ERR + 4 - OFF_CTR, st) != cudaSuccess) return HSK_ECUDA;
    k_noalloc_key_base<<<1, 32, 0, st>>>(reinterpret_cast<unsigned long long*>(key_base), n);
    hsk::launch_digit_hist(d_keys, key_words, n, hist, P, num_sms * 4, st);
    hsk::launch_digit_offsets_seg(hist, key_base, doff, P, 1, st);
    if (cudaGetLastError() != cudaSuccess) return HSK_ECUDA;  // a launch of this call failed
    void *src = d_keys, *dst = alt;
    for (int p = 0; p < P; ++p) {
        // the status words were zeroed above, so pass p may use epoch p + 1
        hsk::launch_onesweep_seg(src, dst, nullptr, nullptr, key_base, 1, (uint32_t)tiles, nullptr, key_words, 8 * p,
                                 doff + (size_t)p * 256, status, ctr + p, (uint32_t)(p + 1), err, st);
        if (cudaGetLastError() != cudaSuccess) return HSK_ECUDA;
        void* t = src;
        src = dst;
        dst = t;
    }
    if (src != d_keys &&
        cudaMemcpyAsync(d_keys, src, n * 8 * (size_t)key_words, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return HSK_ECUDA;
    int herr = 0;
    if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return HSK_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HSK_ECUDA;
    if (herr == HSK_DERR_TIMEOUT) return HSK_ETIMEOUT;
    return herr ? HSK_ECUDA : HSK_OK;
}
