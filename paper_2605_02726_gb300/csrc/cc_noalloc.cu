// coolchic_rate_distortion_noalloc: the rate-distortion evaluation of coolchic_rate_distortion for
// callers that cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc while it runs -- for example a process whose
// device memory is entirely owned by its own pool (a serving process that reserves the HBM up
// front and forbids third-party allocations), or code invoked while another thread of the same
// process holds a CUDA stream in global-mode capture, where cudaMalloc is an illegal call.  Such a
// caller cannot obtain the workspace the other entry points take.  This entry point takes only
// inputs and the output and uses a fixed scratch area compiled into the library instead.
//
// The scratch is a file-scope __device__ array of kNoAllocBytes (32 MiB).  Every GPU on which the
// library is loaded holds it until the process exits.  Host code cannot use the array's name as a
// device address (it names a host-side shadow), so the device address is obtained once per device
// with cudaGetSymbolAddress, on the first call made with that device current; make that first call
// before any stream capture begins.  All calls share the array: two calls that overlap on the GPU
// (different streams, or different host threads) race and may return wrong results.  Every byte
// a call reads is first written by the same call, so nothing has to be cleared between calls.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/coolchic.h"
#include "cc_kernels.h"

namespace cc {
namespace {

constexpr size_t kNoAllocBytes = (size_t)32 << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_na_mu;
std::vector<void*> g_na_ptr;  // device address of the scratch, per device (null until set up)

size_t take(size_t& off, size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
}

// Forward-only layout: y~, the upsampled grids, t, the per-CTA partials and one record (three
// doubles: loss, rate, distortion), whose address goes to *rd.
size_t layout(const cc_arch_t* a, char* base, Work* out, double** rd) {
    Work w;
    std::memset(&w, 0, sizeof(w));
    w.g = make_geom(a->H, a->W);
    w.N = w.g.off[kL];
    w.HW = (int64_t)a->H * a->W;
    w.n_cta_arm = arm_grid(w.N, w.g.nh > 0);
    const int64_t tiles = conv_tiles(a->H, a->W), cap = 2 * (int64_t)num_sms();
    w.n_cta_conv = (int)(tiles < cap ? tiles : cap);
    size_t off = 0;
    const size_t F = sizeof(float);
    const size_t o_yt = take(off, (size_t)w.N * F);
    size_t o_up[kL] = {0};
    for (int m = 1; m <= kL - 2; ++m) o_up[m] = take(off, (size_t)(kL - 1 - m) * w.g.h[m] * w.g.w[m] * F);
    const size_t o_t = take(off, (size_t)3 * w.HW * F);
    const size_t o_rp = take(off, (size_t)w.n_cta_arm * sizeof(double));
    const size_t o_sp = take(off, (size_t)w.n_cta_conv * sizeof(double));
    const size_t o_rd = take(off, 3 * sizeof(double));
    if (base && out) {
        w.yt = (float*)(base + o_yt);
        for (int m = 1; m <= kL - 2; ++m) w.up[m] = (float*)(base + o_up[m]);
        w.t = (float*)(base + o_t);
        w.rate_part = (double*)(base + o_rp);
        w.se_part = (double*)(base + o_sp);
        *out = w;
        *rd = (double*)(base + o_rd);
    }
    return off;
}

}  // namespace
}  // namespace cc

using namespace cc;

extern "C" int coolchic_rate_distortion_noalloc(const cc_arch_t* arch, const cc_hparams_t* hp, const float* image,
                                                const float* latents, const float* params, int64_t step,
                                                int32_t relax, cc_rd_t* rd_out, void* stream) {
    if (!arch) return set_error(CC_ERR_ARG, "arch is NULL");
    cc_arch_t ref;
    if (coolchic_arch_init(&ref, arch->H, arch->W) != CC_OK) return CC_ERR_ARG;  // message already set
    ref.H = arch->H;
    ref.W = arch->W;
    if (std::memcmp(&ref, arch, sizeof(ref)) != 0)
        return set_error(CC_ERR_UNSUPPORTED, "rate_distortion_noalloc: only the architecture of coolchic_arch_init is built");
    if (!hp || !std::isfinite(hp->lambda) || hp->lambda < 0.f)
        return set_error(CC_ERR_ARG, "rate_distortion_noalloc: hparams NULL or lambda not finite and >= 0");
    if (const int rc = validate_hparams(hp)) return rc;
    if (!image || !latents || !params || !rd_out)
        return set_error(CC_ERR_ARG, "rate_distortion_noalloc: NULL image, latents, params or rd_out");
    if (relax < 0 || relax > 2) return set_error(CC_ERR_ARG, "rate_distortion_noalloc: relax must be 0, 1 or 2");
    if (step < 0 || step > 0x7fffffffLL) return set_error(CC_ERR_ARG, "rate_distortion_noalloc: step outside 0..2^31-1");
    const size_t need = layout(arch, nullptr, nullptr, nullptr);
    if (need > kNoAllocBytes)
        return set_error(CC_ERR_WORKSPACE,
                         "rate_distortion_noalloc: a %d x %d image needs %zu bytes of scratch, the built-in limit is "
                         "%zu bytes (about 1.4 million pixels: 1024 x 1024 fits); use coolchic_rate_distortion with a workspace",
                         arch->H, arch->W, need, kNoAllocBytes);
    // SM count and kernel attributes of this device, as every other entry point sets them up first
    // (this allocates nothing)
    if (const int rc = device_setup_checked()) return rc;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(CC_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if ((int)g_na_ptr.size() <= dev) g_na_ptr.resize(dev + 1, nullptr);
        if (!g_na_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // this device is current
            if (e != cudaSuccess || !p)
                return set_error(CC_ERR_CUDA, "cudaGetSymbolAddress of the scratch: %s", cudaGetErrorString(e));
            g_na_ptr[dev] = p;
        }
        base = g_na_ptr[dev];
    }
    Work w;
    double* rd_dev = nullptr;
    layout(arch, (char*)base, &w, &rd_dev);
    cudaStream_t s = (cudaStream_t)stream;
    Hp h;
    h = hp_from(hp);
    launch_relax(w, latents, nullptr, step, h, relax, s);
    launch_arm(w, params, PASS_FWD, 0.f, s);
    launch_up_forward(w, params, kUpArmLo - 1, s);
    launch_syn_forward(w, params, PASS_FWD, s);
    launch_conv(w, params, image, PASS_FWD, 0.f, nullptr, s);
    launch_finish(w, h, 1, 1, rd_dev, nullptr, 0, 0, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(CC_ERR_CUDA, "rate_distortion_noalloc launch: %s", cudaGetErrorString(e));
    e = cudaMemcpyAsync(rd_out, rd_dev, sizeof(cc_rd_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(CC_ERR_CUDA, "rate_distortion_noalloc readback: %s", cudaGetErrorString(e));
    return CC_OK;
}
