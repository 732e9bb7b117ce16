// tl_host_alloc / tl_host_free: page-locked host memory for state copies.
//
// Host memory pinned in base pages (what cudaHostAlloc returns) needs one
// address translation per page for the device's copies; on transparent huge
// pages one translation covers a whole huge page.  This allocator maps
// anonymous memory, asks for transparent huge pages (madvise), faults every
// page in, and registers the range with CUDA (cudaHostRegister), which pins
// it.  Where the kernel grants no huge pages the memory is still pinned and
// correct.  Measured copy rates of such buffers against cudaHostAlloc ones
// varied from one host to the next (at the link's full rate in every repeat
// where cudaHostAlloc buffers dipped, and the other way round elsewhere), so
// this is an option for callers, not a guarantee of the link's rate.
#include <stdint.h>
#include <stdio.h>
#include <sys/mman.h>
#include <unistd.h>

#include <map>
#include <mutex>

#include "tl_internal.cuh"

namespace {

struct Mapping {
    void *base;  // what mmap returned
    size_t len;  // what was mapped
};
std::mutex g_host_mu;
std::map<void *, Mapping> g_host;  // pointer handed out -> its mapping

// The PMD-level transparent huge page size (2 MiB with 4 KiB base pages,
// 512 MiB with 64 KiB ones); 0 when the kernel does not say.
size_t huge_page_bytes()
{
    static size_t cached = [] {
        size_t v = 0;
        if (FILE *f = fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
            unsigned long long x = 0;
            if (fscanf(f, "%llu", &x) == 1) v = (size_t)x;
            fclose(f);
        }
        return v;
    }();
    return cached;
}

int fail(int code, const char *msg, const char *detail = "") { return tl::set_error(code, msg, detail); }

}  // namespace

extern "C" {

int tl_host_alloc(size_t bytes, void **out)
{
    tl::set_error(TL_OK, "", "");
    if (!out) return fail(TL_EINVAL, "NULL out");
    *out = nullptr;
    if (bytes == 0) return fail(TL_EINVAL, "bytes must be > 0");
    const size_t page = (size_t)sysconf(_SC_PAGESIZE);
    const size_t huge = huge_page_bytes();
    // huge-page alignment (start and length) only for buffers of at least one huge page
    const size_t align = (huge >= page && bytes >= huge) ? huge : page;
    const size_t len = (bytes + align - 1) / align * align;
    const size_t map_len = len + (align > page ? align : 0);
    if (len < bytes || map_len < len) return fail(TL_EINVAL, "size overflows");
    void *base = mmap(nullptr, map_len, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (base == MAP_FAILED) return fail(TL_ENOMEM, "mmap of the host buffer failed");
    char *p = reinterpret_cast<char *>(((uintptr_t)base + align - 1) / align * align);
    if (align > page) madvise(p, len, MADV_HUGEPAGE);  // advice only: failure leaves base pages
    volatile char *touch = p;
    for (size_t off = 0; off < len; off += page) touch[off] = 0;  // fault in under the advice
    const cudaError_t e = cudaHostRegister(p, len, cudaHostRegisterDefault);
    if (e != cudaSuccess) {
        munmap(base, map_len);
        return fail(TL_ECUDA, "cudaHostRegister: ", cudaGetErrorString(e));
    }
    {
        std::lock_guard<std::mutex> lock(g_host_mu);
        g_host[p] = Mapping{base, map_len};
    }
    *out = p;
    return TL_OK;
}

int tl_host_free(void *ptr)
{
    tl::set_error(TL_OK, "", "");
    if (!ptr) return TL_OK;
    Mapping m;
    {
        std::lock_guard<std::mutex> lock(g_host_mu);
        auto it = g_host.find(ptr);
        if (it == g_host.end()) return fail(TL_EINVAL, "pointer was not returned by tl_host_alloc (or already freed)");
        m = it->second;
        g_host.erase(it);
    }
    const cudaError_t e = cudaHostUnregister(ptr);
    munmap(m.base, m.len);
    if (e != cudaSuccess) return fail(TL_ECUDA, "cudaHostUnregister: ", cudaGetErrorString(e));
    return TL_OK;
}

}  // extern "C"
