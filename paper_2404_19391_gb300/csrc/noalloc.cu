// zs_decompress_noalloc: zs_decompress for callers that cannot allocate memory.
//
// Some callers cannot let a library allocate: their device memory is entirely reserved by another
// allocator (a framework's caching allocator that has already claimed the free HBM, a fixed arena in an
// embedded service), or they run latency-critical loops where cudaMalloc / cudaFree / cudaMallocHost
// would implicitly synchronise the device. This entry point runs the same decompression kernel as
// zs_decompress but takes its scratch (the look-back records of the tiles and the result words) from a
// fixed array compiled into the library, and copies the result into the caller's zs_result itself.
// It calls no cudaMalloc, cudaFree, cudaMallocHost or other allocating routine.
//
// The array is kNoAllocScratchBytes (8 MiB) of device memory that every GPU loading the library holds
// until the process exits. Every call shares it; calls whose work overlaps on the GPU (from several
// host threads or streams at once) race on it and must be serialised by the caller.
#include "zs_common.cuh"

namespace zs {

namespace {

constexpr size_t kNoAllocScratchBytes = 8u << 20;

// The scratch itself. In host code this name is only a host-side stand-in for the device array, never
// a device address: the kernel gets the address returned by cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// The array's device address on the current device. It is looked up on every call rather than cached:
// after cudaDeviceReset the module is loaded again and a cached address would be stale. Once the module
// is loaded the lookup allocates nothing.
zs_status scratch_address(void **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "zs_decompress_noalloc: cudaGetSymbolAddress");
    *out = p;
    return ZS_OK;
}

}  // namespace
}  // namespace zs

extern "C" zs_status zs_decompress_noalloc(const zs_dict *d, const uint8_t *d_in, size_t in_len, uint8_t *d_out,
                                          size_t out_cap, zs_result *res, void *stream)
{
    zs::clear_error();
    if (!d || !res || (!d_in && in_len) || (!d_out && out_cap)) {
        zs::set_error("zs_decompress_noalloc: NULL argument");
        return ZS_ERR_INVALID_ARG;
    }
    res->out_len = res->n_lines = res->err_offset = 0;
    const uint64_t max_tiles = (zs::kNoAllocScratchBytes - sizeof(zs::DevResult)) / sizeof(zs::TileState);
    const uint64_t ntiles = zs::decompress_tiles(in_len);
    if (ntiles > max_tiles) {
        zs::set_error("zs_decompress_noalloc: input of " + std::to_string(in_len) + " bytes needs " +
                      std::to_string(ntiles) + " tile records; the fixed 8 MiB scratch holds " +
                      std::to_string(max_tiles) + " (use zs_decompress for larger inputs)");
        return ZS_ERR_INVALID_ARG;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return zs::cuda_fail(e, "zs_decompress_noalloc: cudaGetDevice");
    if (dev != d->device) {
        zs::set_error("zs_decompress_noalloc: dictionary was loaded on another device");
        return ZS_ERR_INVALID_ARG;
    }
    if (in_len == 0) return ZS_OK;
    void *scratch = nullptr;
    zs_status st = zs::scratch_address(&scratch);
    if (st != ZS_OK) return st;

    cudaStream_t s = (cudaStream_t)stream;
    zs::DevResult *dr = reinterpret_cast<zs::DevResult *>(scratch);
    zs::TileState *tiles = reinterpret_cast<zs::TileState *>(dr + 1);
    // the array keeps the previous call's contents: the counters and look-back records start at zero
    e = cudaMemsetAsync(scratch, 0, sizeof(zs::DevResult) + ntiles * sizeof(zs::TileState), s);
    if (e == cudaSuccess) e = zs::launch_decompress_single(d, d_in, in_len, d_out, out_cap, dr, tiles, s);
    zs::DevResult r{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&r, dr, sizeof r, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return zs::cuda_fail(e, "zs_decompress_noalloc");
    // the same order as zs_decompress: on a timeout *res stays zero
    if (r.status & zs::kStTimeout) {
        zs::set_error("zs_decompress_noalloc: a device-side wait expired");
        return ZS_ERR_TIMEOUT;
    }
    res->out_len = r.out_len;
    res->n_lines = r.n_lines;
    if (r.status & zs::kStMalformed) {
        res->err_offset = ~r.err_key;
        zs::set_error("zs_decompress_noalloc: malformed input at byte " + std::to_string(res->err_offset));
        return ZS_ERR_MALFORMED;
    }
    if (r.out_len > out_cap) {
        zs::set_error("zs_decompress_noalloc: output buffer too small");
        return ZS_ERR_CAPACITY;
    }
    return ZS_OK;
}

extern "C" size_t zs_decompress_noalloc_limit(void)
{
    const uint64_t max_tiles = (zs::kNoAllocScratchBytes - sizeof(zs::DevResult)) / sizeof(zs::TileState);
    return (size_t)(max_tiles * zs::decompress_tile_bytes());
}
