// H application for callers that cannot allocate device memory.
//
// Some callers of this library run where cudaMalloc is off limits: under an allocator that owns
// all device memory (a framework's caching pool, which would see its budget broken by an
// allocation it does not know about), or in a service whose device memory budget is fixed at
// start-up. For them wdf_apply_hamiltonian_noalloc() computes the same H x as
// wdf_apply_hamiltonian() but takes every temporary from one file-scope device array of
// WDF_NOALLOC_SCRATCH_BYTES bytes. That array exists on every GPU that loads the library, for the
// life of the process. Nothing here calls cudaMalloc, cudaFree or any allocating routine.
//
// Host code cannot use the array's name as a device address (in host code it names a host-side
// stand-in), so the first call on each device looks the address up with cudaGetSymbolAddress
// while that device is current and caches it; that first call should therefore happen before any
// stream capture. Every call on a device reuses the same array, which keeps the previous call's
// contents: the parts that must start at zero are cleared on each call, and two calls whose GPU
// work overlaps in time (different streams, no ordering) race on the array. The whole input is
// copied into the array before the first output element is written, so out may equal in.
#include <cstring>
#include <mutex>

#include "engine.cuh"

namespace wdf {

static __device__ __align__(256) unsigned char g_noalloc_scratch[WDF_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mutex;
static void *g_noalloc_ptr[64] = {nullptr};

// device address of the scratch array on the current device (looked up once per device)
static unsigned char *noalloc_base(int device) {
  if (device < 0 || device >= 64) throw ApiFailure(WDF_EINVAL, "device ordinal out of range for the static scratch");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) throw CudaFailure(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
    g_noalloc_ptr[device] = p;
  }
  return static_cast<unsigned char *>(g_noalloc_ptr[device]);
}

static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// the caller's buffers must be device (or managed) memory of the context's GPU
static void check_device_pointer(const void *p, int device, const char *name) {
  cudaPointerAttributes a{};
  const cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    throw ApiFailure(WDF_EINVAL, std::string(name) + " is not a pointer the CUDA runtime knows");
  }
  if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != device)
    throw ApiFailure(WDF_EINVAL, std::string(name) + " must point to device memory of the context's GPU");
}

}  // namespace wdf

using namespace wdf;

extern "C" int wdf_apply_hamiltonian_noalloc(wdf_ctx *c, int nvec, const double *in, double *out) {
  if (!c) return WDF_EINVAL;
  if (c->failed) {
    c->err = "context unusable after an earlier CUDA failure";
    return WDF_ESTATE;
  }
  try {
    if (nvec < 0 || (nvec > 0 && (!in || !out))) throw ApiFailure(WDF_EINVAL, "bad nvec or NULL buffer");
    if (nvec == 0) return WDF_OK;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) throw CudaFailure(e, "cudaSetDevice", __FILE__, __LINE__);
    check_device_pointer(in, c->device, "in");
    check_device_pointer(out, c->device, "out");
    const Geo &g = c->geo;
    cudaStream_t st = c->st;
    const int npair = (nvec + 1) / 2;
    const int M = c->nproj;
    // carve the array: X, Y (internal vectors), column buffer, projections, split sums, zero shifts
    const size_t bx = align256(sizeof(cplx<double>) * (size_t)nvec * g.ld);
    const size_t bcb = align256(sizeof(cplx<double>) * (size_t)npair * g.n3 * g.ldcb);
    const size_t bs = align256(sizeof(double) * (size_t)std::max(M, 1) * nvec);
    const size_t gwd = gram_work_doubles(g, M, nvec, nvec);
    const size_t bgw = align256(sizeof(double) * std::max<size_t>(gwd, 1));
    const size_t bz = align256(sizeof(double) * (size_t)nvec);
    const size_t need = 2 * bx + bcb + bs + bgw + bz;
    if (need > (size_t)WDF_NOALLOC_SCRATCH_BYTES)
      throw ApiFailure(WDF_EINVAL, "wdf_apply_hamiltonian_noalloc needs " + std::to_string(need) + " bytes of scratch for " +
                                       std::to_string(nvec) + " vectors; the static array holds " +
                                       std::to_string((size_t)WDF_NOALLOC_SCRATCH_BYTES) + " (use fewer vectors per call)");
    unsigned char *base = noalloc_base(c->device);
    cplx<double> *X = reinterpret_cast<cplx<double> *>(base);
    cplx<double> *Y = reinterpret_cast<cplx<double> *>(base + bx);
    cplx<double> *cb = reinterpret_cast<cplx<double> *>(base + 2 * bx);
    double *S = reinterpret_cast<double *>(base + 2 * bx + bcb);
    double *gw = reinterpret_cast<double *>(base + 2 * bx + bcb + bs);
    double *zs = reinterpret_cast<double *>(base + 2 * bx + bcb + bs + bgw);
    // the padding of X and the shifts must be zero; everything else is written before it is read
    WDF_CUDA_TRY(cudaMemsetAsync(X, 0, bx, st));
    WDF_CUDA_TRY(cudaMemsetAsync(zs, 0, bz, st));
    launch_ext_to_int(in, nvec, c->npw_h, c->t_emap.as<int>(), c->t_emap2.as<int>(), c->t_econj.as<int>(), nullptr, X, g.ld, st);
    // H x = 1/2|G|^2 x + fft_n(V_loc ifft(x)) + sum_j beta_j D_j <beta_j, x>
    launch_zpass_g2r<double>(c->f64, X, nvec, cb, st);
    PlaneArgs<double> pa;
    pa.cb = cb;
    pa.field = c->vloc64.as<double>();
    launch_plane<double>(c->f64, OP_VLOC, npair, pa, st);
    EpiArgs<double> ea;
    ea.Y = Y;
    ea.X = X;
    ea.shift = zs;
    ea.scale = 1.0 / (double)c->ngrid;
    launch_zpass_r2g<double>(c->f64, EPI_HSHIFT, cb, nvec, ea, st);
    if (M > 0) {
      launch_gram<double>(g, c->U64.as<cplx<double>>(), M, X, nvec, S, nvec, gw, bgw / sizeof(double), st);
      launch_lincomb<double>(g, Y, nvec, c->U64.as<cplx<double>>(), M, S, nvec, c->lrd.as<double>(), 1.0, st);
    }
    launch_int_to_ext(Y, nvec, g.ld, c->npw_h, c->t_emap.as<int>(), c->t_econj.as<int>(), out, st);
    WDF_CUDA_TRY(cudaStreamSynchronize(st));
    return WDF_OK;
  } catch (const ApiFailure &f) {
    c->err = f.msg;
    return f.code;
  } catch (const CudaFailure &f) {
    c->err = std::string("CUDA error ") + cudaGetErrorName(f.err) + " in " + f.what;
    c->failed = true;
    return WDF_ECUDA;
  } catch (...) {
    c->err = "unexpected C++ exception";
    return WDF_EINVAL;
  }
}
