// rx_kk_field_noalloc: the Kramers-Kronig front end (12-bit unpack, overlap-save
// Hilbert FFT, field sqrt(I) exp(j phi)) for callers that cannot allocate device
// memory.  All scratch lives in one file-scope device array of fixed size; the
// caller passes only the input and the output.  See include/rx.h.
#include <math.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include <cuda_runtime.h>

#include "rx_internal.cuh"

using namespace rxk;

namespace {

constexpr long long kNaMaxSamples = 1LL << 19;          // largest buffer one call accepts
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// byte layout of the scratch array:
//   tables   per FFT length (4096, 65536) a block [ln table | factored W_N | factored W_{N/16}]
//   hist     the packed history the front end is handed; on a stream's first buffer it
//            is never read for values (samples before the stream are the first sample
//            replicated), so it only has to be a valid region of ols_n * 3 / 2 bytes
//   fft      the two-block complex FFT rows, at most 2^19 complex values
//   E        the field [kEHist history | buffer]
//   state    the front end's reduction state (carrier sums and their ticket)
constexpr int kNaSizes = 2;
constexpr size_t kTabBytes = 4096 * sizeof(float) + 1024 * sizeof(float2);   // >= one block
constexpr size_t kOffTw = 0;
constexpr size_t kOffHist = align_up(kOffTw + kNaSizes * kTabBytes);
constexpr size_t kHistBytes = (size_t)65536 * 3 / 2;
constexpr size_t kOffFft = align_up(kOffHist + kHistBytes);
constexpr size_t kFftBytes = 4u << 20;                   // two-block complex FFT rows
constexpr size_t kOffE = align_up(kOffFft + kFftBytes);
constexpr size_t kEBytes = (size_t)(kEHist + kNaMaxSamples) * sizeof(float2);
constexpr size_t kOffState = align_up(kOffE + kEBytes);
constexpr size_t kScratchBytes = align_up(kOffState + sizeof(DevState));

// One scratch region per GPU that loads the library (held until the process exits).
// Every call uses it, so calls that overlap on the GPU race with each other.
static __device__ __align__(256) unsigned char g_na_scratch[kScratchBytes];

// index of the table block of an FFT length (4096 or 65536)
int tab_index(int n) { return n == 4096 ? 0 : 1; }

// per-device set-up: device address of the scratch array and the uploaded tables.
// The first call on a device does it under a lock, so host threads that make their
// first calls at the same time do it once; later calls only read the published flag.
constexpr int kMaxDevices = 64;
unsigned char *g_dev_ptr[kMaxDevices];
std::atomic<bool> g_ready[kMaxDevices];
std::mutex g_setup_mu;

cudaError_t setup_device(int dev, cudaStream_t st, unsigned char **out)
{
    if (g_ready[dev].load(std::memory_order_acquire)) {
        *out = g_dev_ptr[dev];
        return cudaSuccess;
    }
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (g_ready[dev].load(std::memory_order_acquire)) {
        *out = g_dev_ptr[dev];
        return cudaSuccess;
    }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess) return e;
    // lookup and twiddle tables of the two FFT lengths, once per device: copied on the
    // caller's stream, which is then synchronised, so the tables are in place before
    // this call's kernels and before any later call on any stream
    static unsigned char blk[kNaSizes * kTabBytes];
    const int sizes[kNaSizes] = {4096, 65536};
    for (int i = 0; i < kNaSizes; i++) {
        unsigned char *b = blk + i * kTabBytes;
        float *ln = (float *)b;
        float2 *t1 = (float2 *)(ln + 4096), *t2 = t1 + kk_tw_entries(sizes[i]);
        kk_host_tables(sizes[i], ln, t1, t2);
    }
    e = cudaMemcpyAsync((unsigned char *)p + kOffTw, blk, sizeof blk, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = (unsigned char *)p;
    g_ready[dev].store(true, std::memory_order_release);
    *out = (unsigned char *)p;
    return cudaSuccess;
}

__global__ void k_na_copy_field(const float2 *__restrict__ src, float2 *__restrict__ dst, long long n)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i];
}

}  // namespace

extern "C" rx_status rx_kk_field_noalloc(const uint8_t *packed12_in, int64_t nsamp, int32_t pack_order,
                                         int32_t ols_n, int32_t ols_v, float *field_out, void *cuda_stream)
{
    if (!packed12_in || !field_out || nsamp <= 0 || nsamp % 32 || nsamp > kNaMaxSamples) return RX_EINVAL;
    if (((uintptr_t)packed12_in) & 15 || ((uintptr_t)field_out) & 7) return RX_EINVAL;
    if (pack_order < 0 || pack_order > 1) return RX_EINVAL;
    if (!(ols_n == 4096 || ols_n == 65536) || ols_v < 64 || ols_v % 64 || ols_v >= ols_n) return RX_EINVAL;
    long long e_k = nsamp - ols_v / 2;
    if (e_k <= 0) return RX_EINVAL;
    KkGeom g;
    memset(&g, 0, sizeof g);
    g.N = ols_n;
    g.V = ols_v;
    g.hop = ols_n - ols_v;
    g.N2 = ols_n / 16;
    g.J = (int)((e_k + g.hop - 1) / g.hop);
    g.npairs = (g.J + 1) / 2;
    g.e_prev = 0;
    g.e_k = e_k;
    g.avail = nsamp;
    g.cbase = -(long long)ols_n;        // stream index of the packed history's first sample
    g.ebase = -kEHist;                  // field: [kEHist history | buffer]
    g.ebase_prev = -kEHist;
    g.sps = 4;
    g.slot = 0;
    size_t need_fft = (size_t)g.npairs * ols_n * sizeof(float2);
    if (need_fft > kFftBytes) return RX_EINVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RX_ECUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned char *base = nullptr;
    if (setup_device(dev, st, &base) != cudaSuccess) return RX_ECUDA;
    const unsigned char *tabb = base + kOffTw + tab_index(ols_n) * kTabBytes;
    KkTables tb;
    tb.lnt = (const float *)tabb;
    tb.twN = (const float2 *)(tb.lnt + 4096);
    tb.twN2 = tb.twN + kk_tw_entries(ols_n);
    const uint8_t *hist = base + kOffHist;
    float2 *fftws = (float2 *)(base + kOffFft);
    float2 *E = (float2 *)(base + kOffE);
    DevState *ds = (DevState *)(base + kOffState);
    // the carrier sums and the last-CTA ticket of their reduction must start at zero
    if (cudaMemsetAsync(ds, 0, sizeof(DevState), st) != cudaSuccess) return RX_ECUDA;
    KkInput kin;
    kin.hist = hist;                        // never read for values: the first call fills the pre-stream
    kin.in = packed12_in;
    kin.hist_next = nullptr;
    kin.hist_bytes = (long long)ols_n * 3 / 2;
    kin.in_bytes = nsamp * 3 / 2;
    kin.order = pack_order;
    kin.first_call = 1;
    kin.lat = nullptr;
    kin.lat_slot = 0;
    const KkSync none = {nullptr, nullptr, nullptr};
    if (launch_kk_front(g, kin, fftws, tb, E, E, ds, st, nullptr, none) != cudaSuccess) return RX_ECUDA;
    unsigned grid = (unsigned)((e_k + 255) / 256);
    k_na_copy_field<<<grid, 256, 0, st>>>(E + kEHist, reinterpret_cast<float2 *>(field_out), e_k);
    if (cudaGetLastError() != cudaSuccess) return RX_ECUDA;
    return RX_OK;
}
