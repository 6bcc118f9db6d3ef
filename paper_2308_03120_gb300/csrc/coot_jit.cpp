// Run-time compilation and caching of the per-tree kernels.
//
// Bandicoot compiles its GPU kernels at run time for the device it finds
// and keeps them in an on-disk cache so that later runs skip the compile
// (Section 3 of arXiv 2308.03120).  The same holds here, per tree: a kernel
// is looked up by a digest of its full source and target architecture in
// an in-memory table, then in the on-disk cache ($COOT_CACHE_DIR, default
// $HOME/.cache/coot-gb300; "off" disables it), and only then compiled with
// NVRTC into a cubin for the device (sm_103a on GB300).  Cache files carry
// a checksum; a file that fails it is ignored and rewritten.
#include <cuda_runtime.h>
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <atomic>
#include <cinttypes>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>

#include "coot_internal.h"

namespace coot {

static std::mutex g_mu;
static std::unordered_map<uint64_t, Compiled> g_kernels;
static Device g_dev;
static bool g_init = false;

const Device& device() { return g_dev; }
bool initialised() { return g_init; }

static std::string fault() {
  const char* f = std::getenv("COOT_FAULT");
  return f ? std::string(f) : std::string();
}

static std::string arch_name(int major, int minor) {
  // architecture-specific targets ("a") exist from compute capability 9.0 on
  return "sm_" + std::to_string(major) + std::to_string(minor) + (major >= 9 ? "a" : "");
}

static std::string cache_dir() {
  const char* d = std::getenv("COOT_CACHE_DIR");
  if (d && std::strcmp(d, "off") == 0) return "";
  if (d && *d) return d;
  const char* home = std::getenv("HOME");
  return std::string(home && *home ? home : "/tmp") + "/.cache/coot-gb300";
}

static void mkdirs(const std::string& path) {
  std::string cur;
  for (size_t i = 0; i < path.size(); ++i) {
    cur += path[i];
    if (path[i] == '/' && cur.size() > 1) mkdir(cur.c_str(), 0755);
  }
  mkdir(path.c_str(), 0755);
}

struct CacheHeader {
  char magic[8];
  uint64_t key;
  uint64_t size;
  uint64_t checksum;
};

static bool read_cache(const std::string& path, uint64_t key, std::string* cubin) {
  FILE* f = std::fopen(path.c_str(), "rb");
  if (!f) return false;
  CacheHeader h;
  bool ok = std::fread(&h, sizeof h, 1, f) == 1 && std::memcmp(h.magic, "COOTCUBN", 8) == 0 &&
            h.key == key && h.size > 0 && h.size < (1ull << 30);
  if (ok) {
    cubin->resize(h.size);
    ok = std::fread(&(*cubin)[0], 1, h.size, f) == h.size;
  }
  std::fclose(f);
  if (ok && fault() == "cache_corrupt") (*cubin)[cubin->size() / 2] ^= 0x5a;
  return ok && fnv1a(cubin->data(), cubin->size()) == h.checksum;
}

static void write_cache(const std::string& path, uint64_t key, const std::string& cubin) {
  static std::atomic<unsigned> serial{0};
  const std::string tmp = path + ".tmp" + std::to_string(getpid()) + "." + std::to_string(serial++);
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return;
  CacheHeader h;
  std::memcpy(h.magic, "COOTCUBN", 8);
  h.key = key;
  h.size = cubin.size();
  h.checksum = fnv1a(cubin.data(), cubin.size());
  bool ok = std::fwrite(&h, sizeof h, 1, f) == 1 && std::fwrite(cubin.data(), 1, cubin.size(), f) == cubin.size();
  ok = (std::fclose(f) == 0) && ok;
  if (ok) {
    std::rename(tmp.c_str(), path.c_str());
  } else {
    std::remove(tmp.c_str());
  }
}

// NVRTC: source -> cubin for `arch`.
static coot_status nvrtc_compile(const std::string& source, const std::string& arch, std::string* cubin) {
  if (fault() == "nvrtc_fail") return fail(COOT_ERR_COMPILE, "NVRTC failure injected by COOT_FAULT=nvrtc_fail");
  nvrtcProgram prog;
  nvrtcResult r = nvrtcCreateProgram(&prog, source.c_str(), "coot_kernel.cu", 0, nullptr, nullptr);
  if (r != NVRTC_SUCCESS) return fail(COOT_ERR_COMPILE, std::string("nvrtcCreateProgram: ") + nvrtcGetErrorString(r));
  const std::string arch_opt = "--gpu-architecture=" + arch;
  const char* opts[] = {arch_opt.c_str(), "-std=c++17", "-lineinfo", "--fmad=true"};
  r = nvrtcCompileProgram(prog, 4, opts);
  if (r != NVRTC_SUCCESS) {
    size_t n = 0;
    nvrtcGetProgramLogSize(prog, &n);
    std::string log(n, '\0');
    if (n) nvrtcGetProgramLog(prog, &log[0]);
    nvrtcDestroyProgram(&prog);
    return fail(COOT_ERR_COMPILE, "NVRTC compile failed (" + arch + "): " + log.substr(0, 4000));
  }
  size_t n = 0;
  r = nvrtcGetCUBINSize(prog, &n);
  if (r != NVRTC_SUCCESS || n == 0) {
    nvrtcDestroyProgram(&prog);
    return fail(COOT_ERR_COMPILE, "NVRTC produced no cubin");
  }
  cubin->resize(n);
  nvrtcGetCUBIN(prog, &(*cubin)[0]);
  nvrtcDestroyProgram(&prog);
  return COOT_OK;
}

coot_status compile_only(const std::string& source, const std::string& arch, size_t* bytes) {
  std::string cubin;
  coot_status s = nvrtc_compile(source, arch, &cubin);
  if (s == COOT_OK && bytes) *bytes = cubin.size();
  return s;
}

coot_status get_kernel(const std::string& source, const KernelSpec& spec, const Compiled** out) {
  std::string arch;
  uint64_t key;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_init) return fail(COOT_ERR_NOT_INIT, "coot_init has not been called");
    arch = arch_name(g_dev.cc_major, g_dev.cc_minor);
    key = fnv1a(source.data(), source.size());
    key = fnv1a(arch.data(), arch.size(), key);
    auto it = g_kernels.find(key);
    if (it != g_kernels.end()) {
      *out = &it->second;
      return COOT_OK;
    }
  }
  // compile without holding the lock, so that threads compile in parallel
  std::string cubin;
  const std::string dir = cache_dir();
  char name[64];
  std::snprintf(name, sizeof name, "/%016" PRIx64 "-%s.cubin", key, arch.c_str());
  const std::string path = dir.empty() ? std::string() : dir + name;
  if (path.empty() || !read_cache(path, key, &cubin)) {
    coot_status s = nvrtc_compile(source, arch, &cubin);
    if (s != COOT_OK) return s;
    if (!path.empty()) {
      mkdirs(dir);
      write_cache(path, key, cubin);
    }
  }
  std::lock_guard<std::mutex> lock(g_mu);
  auto again = g_kernels.find(key);
  if (again != g_kernels.end()) {  // another thread finished first
    *out = &again->second;
    return COOT_OK;
  }
  cudaLibrary_t lib;
  cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e != cudaSuccess) return fail(COOT_ERR_CUDA, std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e));
  cudaKernel_t k;
  e = cudaLibraryGetKernel(&k, lib, entry_name(spec));
  if (e != cudaSuccess) return fail(COOT_ERR_CUDA, std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(e));
  Compiled c;
  c.kernel = (void*)k;
  cudaFuncAttributes attr;
  if (cudaFuncGetAttributes(&attr, (const void*)k) == cudaSuccess) c.num_regs = attr.numRegs;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)k, spec.block, 0) != cudaSuccess || nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  c.max_blocks_per_sm = nb;
  auto ins = g_kernels.emplace(key, c);
  *out = &ins.first->second;
  return COOT_OK;
}

// Calls after the first with the same tree and kernel shape skip source
// generation: the kernel is found by a digest of the tree bytes and of
// every field of the spec.
static std::mutex g_fast_mu;
static std::unordered_map<uint64_t, const Compiled*> g_fast;

static uint64_t spec_key(const Tree& t, const KernelSpec& s) {
  const int64_t f[] = {s.kind, s.in_dtype[0], s.in_dtype[1], s.in_dtype[2], s.in_dtype[3], s.out_dtype,
                       s.store, (int64_t)s.heads, s.vec, s.unroll, s.block, s.nc, g_dev.id, s.n_trees,
                       (int64_t)s.tree_heads[0], (int64_t)s.tree_heads[1], (int64_t)s.tree_heads[2],
                       (int64_t)s.tree_heads[3], s.tree_out[0], s.tree_out[1], s.tree_out[2], s.tree_out[3],
                       s.tree_cs[0], s.tree_cs[1], s.tree_cs[2], s.tree_cs[3], s.tree_rs[0], s.tree_rs[1],
                       s.tree_rs[2], s.tree_rs[3], s.min_blocks, s.prefetch};
  uint64_t h = t.hash;
  for (int k = 0; k < s.n_trees && s.trees; ++k) h = fnv1a(&s.trees[k].hash, sizeof s.trees[k].hash, h);
  return fnv1a(f, sizeof f, h);
}

coot_status kernel_for(const Tree& t, const KernelSpec& spec, const Compiled** out) {
  const uint64_t key = spec_key(t, spec);
  {
    std::lock_guard<std::mutex> lock(g_fast_mu);
    auto it = g_fast.find(key);
    if (it != g_fast.end()) {
      *out = it->second;
      return COOT_OK;
    }
  }
  coot_status s = get_kernel(generate_source(t, spec), spec, out);
  if (s != COOT_OK) return s;
  std::lock_guard<std::mutex> lock(g_fast_mu);
  g_fast[key] = *out;
  return COOT_OK;
}

void drop_kernels() {
  {
    std::lock_guard<std::mutex> lock(g_fast_mu);
    g_fast.clear();
  }
  std::lock_guard<std::mutex> lock(g_mu);
  g_kernels.clear();  // library handles stay loaded until the process exits
}

coot_status init_device(int dev, unsigned flags) {
  std::lock_guard<std::mutex> lock(g_mu);
  cudaError_t e = cudaSetDevice(dev);
  if (e != cudaSuccess) return fail(COOT_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return fail(COOT_ERR_CUDA, std::string("cudaGetDeviceProperties: ") + cudaGetErrorString(e));
  if (g_init && g_dev.id != dev) {
    std::lock_guard<std::mutex> fast(g_fast_mu);
    g_fast.clear();
    g_kernels.clear();
  }
  g_dev.id = dev;
  g_dev.sm_count = prop.multiProcessorCount;
  g_dev.cc_major = prop.major;
  g_dev.cc_minor = prop.minor;
  g_dev.max_threads_per_sm = prop.maxThreadsPerMultiProcessor;
  g_init = true;
  if (flags & 1u) {
    std::fprintf(stderr, "coot: device %d %s, %d SMs, %s, L2 %d MiB, kernel cache %s\n", dev, prop.name,
                 prop.multiProcessorCount, arch_name(prop.major, prop.minor).c_str(), prop.l2CacheSize >> 20,
                 cache_dir().empty() ? "off" : cache_dir().c_str());
  }
  return COOT_OK;
}

}  // namespace coot
