// Runtime compilation of user kernels (Sec. 3.5 "Runtime Kernel Compilation").
//
// The user writes the kernel body in the paper's convention (Listing 2): a
// __device__ function whose first parameter is the virtual block index and
// whose array parameters are view types indexed with GLOBAL indices:
//     __device__ void name(dim3 virtBlockIdx, <parameters in declaration order>)
// value parameters: int64_t (integer) or double (float); arrays:
// lightning::Vector<T> (1-D, v[i]), Matrix<T> (2-D, m(i, j) or m[i][j]) and
// Tensor<T> (3-D, t(k, i, j)), T = float, double, unsigned short (bf16 bits),
// unsigned char or unsigned int.  lightning::div_rn<C>(float) and
// div4_rn<C>(float4) divide by a small integer constant with IEEE rounding in
// a few instructions (the built-in stencils' method).
//
// Like the generated wrapper of Listing 3, the library adds a __global__
// wrapper that turns the physical block index into the virtual one and builds
// the views from the chunk views (base pointer with the chunk offset already
// subtracted), then calls the user function.  The wrapper reads the same task
// table as the built-in kernels, so one launch runs every superblock of a
// group.  Source and wrapper are compiled by NVRTC for sm_103a and loaded
// with cudaLibraryLoadData.  NVRTC is opened at run time, so the engine loads
// without it; registering a source kernel then reports LT_ERR_UNSUPPORTED.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "core.hpp"
#include "kernels.cuh"
#include "userkernel.hpp"

namespace lt {
namespace {

struct Nvrtc {
    bool ok = false;
    nvrtcResult (*create)(nvrtcProgram *, const char *, const char *, int, const char *const *, const char *const *);
    nvrtcResult (*compile)(nvrtcProgram, int, const char *const *);
    nvrtcResult (*log_size)(nvrtcProgram, size_t *);
    nvrtcResult (*log)(nvrtcProgram, char *);
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t *);
    nvrtcResult (*cubin)(nvrtcProgram, char *);
    nvrtcResult (*destroy)(nvrtcProgram *);
};

Nvrtc &nvrtc() {
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so"};
        void *h = nullptr;
        for (const char *nm : names)
            if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) return;
        n.create = (decltype(n.create))dlsym(h, "nvrtcCreateProgram");
        n.compile = (decltype(n.compile))dlsym(h, "nvrtcCompileProgram");
        n.log_size = (decltype(n.log_size))dlsym(h, "nvrtcGetProgramLogSize");
        n.log = (decltype(n.log))dlsym(h, "nvrtcGetProgramLog");
        n.cubin_size = (decltype(n.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
        n.cubin = (decltype(n.cubin))dlsym(h, "nvrtcGetCUBIN");
        n.destroy = (decltype(n.destroy))dlsym(h, "nvrtcDestroyProgram");
        n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy;
    });
    return n;
}

const char *ctype(int dtype) {
    switch (dtype) {
        case LT_F32: return "float";
        case LT_BF16: return "unsigned short";
        case LT_U8: return "unsigned char";
        case LT_F64: return "double";
        default: return "unsigned int";
    }
}

}  // namespace

// The replica phase of the wrapper: after the CTA's last block, one thread
// per CTA adds the CTA to the grid barrier (a device counter) and waits until
// the counter reaches the launch's target, which the host sets to the number
// of arrivals once every CTA of this launch has arrived; the launch is
// cooperative, so all its CTAs are resident together.  The wait is bounded
// (2 s, %globaltimer): on expiry the CTA records 0x6750 in the error word and
// leaves the replicas as they were.  Then the CTAs copy the replica boxes
// (each LtCopy a box of the written chunk and its replica in a neighbouring
// chunk), in units of 32 consecutive elements of a box (LtUnit: box, first
// element), one element per thread, reading through L2: the written cells
// come from other SMs.
// Correctly rounded division by a small integer constant for user bodies,
// the method of the built-in stencils (Markstein's correction step, P.
// Markstein, IBM J. Res. Dev. 34(1), 1990): with y = RN(1/C), q0 = RN(a*y),
// r = fma(-q0, C, a) is exact and RN(q0 + r*y) is the IEEE quotient for
// 1e-30 <= |a| <= 1e30; other values take the IEEE division.  div4_rn<C>
// tests the range once for four values (the largest magnitude taken
// NaN-propagating, so a NaN fails the test).
static const char *kDivHelpers =
    "template <int C> __device__ __forceinline__ float div_rn(float a) {\n"
    "  const float y = 1.0f / (float)C, m = fabsf(a);\n"
    "  if (!(m >= 1e-30f && m <= 1e30f)) return __fdiv_rn(a, (float)C);\n"
    "  const float q0 = __fmul_rn(a, y);\n"
    "  return __fmaf_rn(__fmaf_rn(-q0, (float)C, a), y, q0);\n"
    "}\n"
    "__device__ __forceinline__ float max_nan(float a, float b) {\n"
    "  float r; asm(\"max.NaN.f32 %0, %1, %2;\" : \"=f\"(r) : \"f\"(a), \"f\"(b)); return r;\n"
    "}\n"
    "template <int C> __device__ __forceinline__ float4 div4_rn(float4 a) {\n"
    "  const float y = 1.0f / (float)C;\n"
    "  const float ax = fabsf(a.x), ay = fabsf(a.y), az = fabsf(a.z), aw = fabsf(a.w);\n"
    "  const float lo = fminf(fminf(ax, ay), fminf(az, aw)), hi = max_nan(max_nan(ax, ay), max_nan(az, aw));\n"
    "  if (!(lo >= 1e-30f && hi <= 1e30f)) return make_float4(div_rn<C>(a.x), div_rn<C>(a.y), div_rn<C>(a.z), div_rn<C>(a.w));\n"
    "  const float qx = __fmul_rn(a.x, y), qy = __fmul_rn(a.y, y), qz = __fmul_rn(a.z, y), qw = __fmul_rn(a.w, y);\n"
    "  return make_float4(__fmaf_rn(__fmaf_rn(-qx, (float)C, a.x), y, qx), __fmaf_rn(__fmaf_rn(-qy, (float)C, a.y), y, qy),\n"
    "                     __fmaf_rn(__fmaf_rn(-qz, (float)C, a.z), y, qz), __fmaf_rn(__fmaf_rn(-qw, (float)C, a.w), y, qw));\n"
    "}\n";

static const char *kReplicaPhase =
    "struct LtUnit { unsigned box, first; };\n"
    "__device__ __forceinline__ unsigned long long lt_gtimer() {\n"
    "  unsigned long long t; asm volatile(\"mov.u64 %0, %%globaltimer;\" : \"=l\"(t)); return t;\n"
    "}\n"
    "__device__ __noinline__ void lt_replicas(const LtCopy *__restrict__ cp, const LtUnit *__restrict__ cu,\n"
    "    unsigned nu, unsigned long long *bar, unsigned long long target, uint32_t *err) {\n"
    "  __shared__ int lt_ok;\n"
    "  __syncthreads();\n"
    "  if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {\n"
    "    __threadfence();\n"
    "    atomicAdd(bar, 1ull);\n"
    "    const unsigned long long t0 = lt_gtimer();\n"
    "    int ok = 1;\n"
    "    for (;;) {\n"
    "      unsigned long long v;\n"
    "      asm volatile(\"ld.acquire.gpu.global.u64 %0, [%1];\" : \"=l\"(v) : \"l\"(bar) : \"memory\");\n"
    "      if (v >= target) break;\n"
    "      if (lt_gtimer() - t0 > 2000000000ull) { atomicCAS(err, 0u, 0x6750u); ok = 0; break; }\n"
    "      __nanosleep(64);\n"
    "    }\n"
    "    __threadfence();\n"
    "    lt_ok = ok;\n"
    "  }\n"
    "  __syncthreads();\n"
    "  if (!lt_ok) return;\n"
    "  const unsigned nth = blockDim.x * blockDim.y * blockDim.z;\n"
    "  const unsigned tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);\n"
    "  const unsigned long long total = (unsigned long long)nu * 32ull;\n"
    "  for (unsigned long long e = (unsigned long long)blockIdx.x * nth + tid; e < total;\n"
    "       e += (unsigned long long)gridDim.x * nth) {\n"
    "    const LtUnit u = cu[e >> 5];\n"
    "    const LtCopy &c = cp[u.box];\n"
    "    const unsigned w0 = (unsigned)(c.hi[0] - c.lo[0] + 1), w1 = (unsigned)(c.hi[1] - c.lo[1] + 1),\n"
    "                   w2 = (unsigned)(c.hi[2] - c.lo[2] + 1);\n"
    "    unsigned l = u.first + (unsigned)(e & 31u);\n"
    "    int64_t g0, g1 = 0, g2 = 0;\n"
    "    if (c.nd == 1) { if (l >= w0) continue; g0 = c.lo[0] + l; }\n"
    "    else if (c.nd == 2) { if (l >= w0 * w1) continue; g0 = c.lo[0] + l / w1; g1 = c.lo[1] + l % w1; }\n"
    "    else { if (l >= w0 * w1 * w2) continue; const unsigned r = l / w2; g2 = c.lo[2] + l % w2;\n"
    "           g1 = c.lo[1] + r % w1; g0 = c.lo[0] + r / w1; }\n"
    "    const int64_t os = g0 * c.src.s[0] + g1 * c.src.s[1] + g2 * c.src.s[2];\n"
    "    const int64_t od = g0 * c.dst.s[0] + g1 * c.dst.s[1] + g2 * c.dst.s[2];\n"
    "    const char *sa = (const char *)(c.src.base + (uint64_t)(os * c.esize));\n"
    "    char *da = (char *)(c.dst.base + (uint64_t)(od * c.esize));\n"
    "    switch (c.esize) {\n"
    "      case 1: *(unsigned char *)da = __ldcg((const unsigned char *)sa); break;\n"
    "      case 2: *(unsigned short *)da = __ldcg((const unsigned short *)sa); break;\n"
    "      case 4: *(unsigned int *)da = __ldcg((const unsigned int *)sa); break;\n"
    "      default: *(unsigned long long *)da = __ldcg((const unsigned long long *)sa); break;\n"
    "    }\n"
    "  }\n"
    "}\n";

std::string user_wrapper_source(const std::string &user, const std::string &name, const std::vector<UserParam> &params) {
    std::ostringstream o;
    o << "typedef long long int64_t;\ntypedef unsigned long long uint64_t;\ntypedef unsigned int uint32_t;\n"
         "typedef int int32_t;\n"
         "namespace lightning {\n"
         "template <typename T> struct Vector {\n"
         "  T *p; int64_t s0;\n"
         "  __device__ T &operator[](int64_t i) const { return p[i * s0]; }\n"
         "  __device__ T &operator()(int64_t i) const { return p[i * s0]; }\n"
         "};\n"
         "template <typename T> struct Matrix {\n"
         "  T *p; int64_t s0, s1;\n"
         "  struct Row { T *p; int64_t s1; __device__ T &operator[](int64_t j) const { return p[j * s1]; } };\n"
         "  __device__ T &operator()(int64_t i, int64_t j) const { return p[i * s0 + j * s1]; }\n"
         "  __device__ Row operator[](int64_t i) const { Row r; r.p = p + i * s0; r.s1 = s1; return r; }\n"
         "};\n"
         "template <typename T> struct Tensor {\n"
         "  T *p; int64_t s0, s1, s2;\n"
         "  __device__ T &operator()(int64_t k, int64_t i, int64_t j) const { return p[k * s0 + i * s1 + j * s2]; }\n"
         "};\n"
      << kDivHelpers << "}  // namespace lightning\n"
         "struct LtView { uint64_t base; int64_t s[3]; int64_t org[3]; int64_t hi[3]; };\n"
         "struct LtTask { int64_t t_lo[3], t_hi[3]; LtView v["
      << LT_MAX_ARRAYS
      << "]; uint32_t cta_begin, cta_count; uint32_t aux[6]; };\n"
         "struct LtParams { int64_t shape["
      << LT_MAX_ARRAYS << "][3]; int32_t nd[" << LT_MAX_ARRAYS
      << "]; int64_t block[3]; double f[4]; int64_t i[4]; uint32_t *err;"
         " int32_t ntasks, variant, red_op, uniform_ctas; const void *reps; uint64_t rep_cells;"
         " uint32_t nreps, rep_ctas; int32_t no_staged, pdl; const void *runits; uint32_t nunits, pad; };\n"
         "static_assert(sizeof(LtView) == "
      << sizeof(DView) << ", \"view layout\");\nstatic_assert(sizeof(LtTask) == " << sizeof(ExecTask)
      << ", \"task layout\");\nstatic_assert(sizeof(LtParams) == " << sizeof(ExecParams) << ", \"params layout\");\n"
      << "struct LtCopy { LtView src, dst; int64_t lo[3], hi[3]; int32_t nd, esize; uint64_t first; };\n"
         "static_assert(sizeof(LtCopy) == "
      << sizeof(CopyPiece) << ", \"copy layout\");\n"
      << kReplicaPhase << "#line 1 \"user_kernel.cu\"\n"
      << user << "\n"
      << "extern \"C\" __global__ void lt_user_wrapper(const LtTask *__restrict__ tasks, LtParams P, unsigned nblocks,\n"
         "    const LtCopy *__restrict__ lt_cp, const LtUnit *__restrict__ lt_cu, unsigned lt_nu,\n"
         "    unsigned long long *lt_bar, unsigned long long lt_target) {\n"
         "  // persistent: each CTA runs the blocks b = blockIdx.x, blockIdx.x + gridDim.x, ... of the launch.\n"
         "  // One thread maps each block to its task and virtual index, one block ahead, into the other of two\n"
         "  // shared slots; the barrier at the top of each block orders the writes and the reads.\n"
         "  __shared__ unsigned lt_maps[2][4];\n"
         "  const bool lt_lead = threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0;\n"
         "  auto lt_find = [&](unsigned b, unsigned *m) {\n"
         "    int lo = 0, hi = P.ntasks - 1;\n"
         "    if (P.uniform_ctas > 0) lo = (int)(b / (unsigned)P.uniform_ctas);\n"
         "    else while (lo < hi) { int mid = (lo + hi + 1) >> 1; if (tasks[mid].cta_begin <= b) lo = mid; else hi = mid - 1; }\n"
         "    const LtTask &tt = tasks[lo];\n"
         "    // first virtual block and the task's extent in blocks along x and y (set by the host)\n"
         "    const unsigned l = b - tt.cta_begin, q = l / tt.aux[3];\n"
         "    m[0] = (unsigned)lo; m[1] = tt.aux[0] + (l - q * tt.aux[3]);\n"
         "    m[2] = tt.aux[1] + q % tt.aux[4]; m[3] = tt.aux[2] + q / tt.aux[4];\n"
         "  };\n"
         "  if (lt_lead && blockIdx.x < nblocks) lt_find(blockIdx.x, lt_maps[0]);\n"
         "  unsigned lt_par = 0;\n"
         "  for (unsigned b = blockIdx.x; b < nblocks; b += gridDim.x, lt_par ^= 1u) {\n"
         "  __syncthreads();\n"
         "  const unsigned *lt_map = lt_maps[lt_par];\n"
         "  const LtTask &t = tasks[lt_map[0]];\n"
         "  dim3 vb(lt_map[1], lt_map[2], lt_map[3]);\n"
         "  if (lt_lead && b + gridDim.x < nblocks) lt_find(b + gridDim.x, lt_maps[lt_par ^ 1u]);\n";
    int slot = 0, fi = 0, ii = 0;
    std::ostringstream args;
    for (size_t p = 0; p < params.size(); ++p) {
        const UserParam &up = params[p];
        args << ", ";
        if (!up.is_array) {
            if (up.dtype == LT_F32)
                args << "P.f[" << fi++ << "]";
            else
                args << "P.i[" << ii++ << "]";
            continue;
        }
        const char *ct = ctype(up.dtype);
        o << "  ";
        if (up.rank == 1)
            o << "lightning::Vector<" << ct << "> a" << slot << "; a" << slot << ".p = (" << ct << " *)t.v[" << slot
              << "].base; a" << slot << ".s0 = t.v[" << slot << "].s[0];\n";
        else if (up.rank == 2)
            o << "lightning::Matrix<" << ct << "> a" << slot << "; a" << slot << ".p = (" << ct << " *)t.v[" << slot
              << "].base; a" << slot << ".s0 = t.v[" << slot << "].s[0]; a" << slot << ".s1 = t.v[" << slot
              << "].s[1];\n";
        else
            o << "lightning::Tensor<" << ct << "> a" << slot << "; a" << slot << ".p = (" << ct << " *)t.v[" << slot
              << "].base; a" << slot << ".s0 = t.v[" << slot << "].s[0]; a" << slot << ".s1 = t.v[" << slot
              << "].s[1]; a" << slot << ".s2 = t.v[" << slot << "].s[2];\n";
        args << "a" << slot;
        slot++;
    }
    // the barrier at the top of the next block also keeps the body's shared memory apart between blocks
    o << "  " << name << "(vb" << args.str() << ");\n  }\n"
      << "  if (lt_nu) lt_replicas(lt_cp, lt_cu, lt_nu, lt_bar, lt_target, P.err);\n}\n";
    return o.str();
}

lt_status compile_user_kernel(const std::string &src, std::vector<char> *cubin, std::string *log) {
    Nvrtc &n = nvrtc();
    if (!n.ok) {
        *log = "NVRTC (libnvrtc.so) could not be opened";
        return LT_ERR_UNSUPPORTED;
    }
    if (const char *dump = std::getenv("LT_NVRTC_DUMP")) {  // debugging aid: the generated source
        if (FILE *f = std::fopen(dump, "w")) {
            std::fwrite(src.data(), 1, src.size(), f);
            std::fclose(f);
        }
    }
    nvrtcProgram prog;
    if (n.create(&prog, src.c_str(), "lightning_user.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        *log = "nvrtcCreateProgram failed";
        return LT_ERR_UNSUPPORTED;
    }
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--fmad=false", "-default-device"};
    nvrtcResult r = n.compile(prog, 4, opts);
    size_t ls = 0;
    n.log_size(prog, &ls);
    std::string lg(ls, '\0');
    if (ls) n.log(prog, &lg[0]);
    *log = lg;
    if (r != NVRTC_SUCCESS) {
        n.destroy(&prog);
        return LT_ERR_COMPILE;
    }
    size_t cs = 0;
    n.cubin_size(prog, &cs);
    cubin->resize(cs);
    n.cubin(prog, cubin->data());
    n.destroy(&prog);
    return LT_OK;
}

namespace k {

// One CTA per virtual block of each task.  aux[0..2] = the task's first
// virtual block, aux[3], aux[4] = its extent in blocks along x and y, so the
// wrapper maps its CTA with two 32-bit divisions.  Virtual block indices are
// dim3 components: every value must fit 32 bits (else the launch is refused).
uint32_t prepare_user(ExecTask *t, int n, ExecParams &p) {
    uint64_t total = 0;
    for (int i = 0; i < n; ++i) {
        uint64_t nb = 1;
        int64_t first[3], ext[3];
        for (int d = 0; d < 3; ++d) {
            const int64_t B = p.block[d] > 0 ? p.block[d] : 1;
            first[d] = t[i].t_lo[d] / B;
            ext[d] = t[i].t_hi[d] / B - first[d] + 1;
            if (t[i].t_hi[d] / B > 0xFFFFFFFFll) return 0xFFFFFFFFu;
            nb *= (uint64_t)ext[d];
        }
        for (int d = 0; d < 3; ++d) t[i].aux[d] = (int32_t)(uint32_t)first[d];
        t[i].aux[3] = (int32_t)(uint32_t)ext[0];
        t[i].aux[4] = (int32_t)(uint32_t)ext[1];
        t[i].cta_begin = (uint32_t)total;
        t[i].cta_count = (uint32_t)nb;
        total += nb;
        if (total >= 0xFFFFFFFFull) return 0xFFFFFFFFu;
    }
    return (uint32_t)total;
}

}  // namespace k
}  // namespace lt
