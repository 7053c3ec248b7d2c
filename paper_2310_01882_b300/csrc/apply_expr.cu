// apply_expr.cu -- the general stencil.apply (Section 2.2): out(x) = an
// expression that reads up to eight input fields at constant offsets, any
// body -- linear or not (the advection's products, quotients, ...).
//
// The expression is translated into the body of a CUDA C kernel (every
// operation an explicitly rounded binary64 intrinsic, in the order of the
// expression's tree, so no multiply-add is fused), compiled at run time for
// the device with NVRTC (loaded on first use, so the library does not
// depend on it otherwise), loaded with cudaLibraryLoadData and cached in the
// context by its source.  The generated kernel is one thread per output
// point, neighbours through L1: bound by the FP64 pipe like any binary64
// stencil on B300, and exactly the expression's binary64 value.
//
// Grammar (whitespace ignored):
//   expr    := term { ('+' | '-') term }
//   term    := unary { ('*' | '/') unary }
//   unary   := '-' unary | primary
//   primary := number | ref | '(' expr ')'
//   ref     := 'a' digit '(' int ',' int ',' int ')'   (input, dx, dy, dz)
//   number  := decimal literal (digits, '.', exponent)
#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace stencil {

namespace {

constexpr int kExprMaxInputs = 8;
constexpr size_t kExprMaxLen = 1 << 16;
constexpr int kExprMaxDepth = 200;

// Recursive-descent translation of an expression into CUDA C.
struct ExprParser {
  const char* s;
  size_t pos = 0;
  int ninputs;
  int radius = 0;
  int depth = 0;
  std::string err;

  void skip() {
    while (s[pos] == ' ' || s[pos] == '\t' || s[pos] == '\n' || s[pos] == '\r') ++pos;
  }
  bool fail(const char* what) {
    if (err.empty()) {
      char b[160];
      snprintf(b, sizeof(b), "apply_expr: %s at offset %zu", what, pos);
      err = b;
    }
    return false;
  }
  bool integer(int* v) {
    skip();
    int sign = 1;
    if (s[pos] == '-' || s[pos] == '+') {
      sign = s[pos] == '-' ? -1 : 1;
      ++pos;
      skip();
    }
    if (s[pos] < '0' || s[pos] > '9') return fail("expected an integer offset");
    long x = 0;
    while (s[pos] >= '0' && s[pos] <= '9') {
      x = x * 10 + (s[pos] - '0');
      if (x > 1000) return fail("offset too large");
      ++pos;
    }
    *v = static_cast<int>(sign * x);
    return true;
  }
  bool expect(char c) {
    skip();
    if (s[pos] != c) {
      char b[40];
      snprintf(b, sizeof(b), "expected '%c'", c);
      return fail(b);
    }
    ++pos;
    return true;
  }
  bool primary(std::string* out) {
    skip();
    const char c = s[pos];
    if (c == '(') {
      ++pos;
      if (!expr(out)) return false;
      return expect(')');
    }
    if (c == 'a') {
      ++pos;
      if (s[pos] < '0' || s[pos] > '9') return fail("expected an input index after 'a'");
      const int idx = s[pos] - '0';
      ++pos;
      if (idx >= ninputs) return fail("input index beyond the inputs given");
      int d[3];
      if (!expect('(') || !integer(&d[0]) || !expect(',') || !integer(&d[1]) || !expect(',') ||
          !integer(&d[2]) || !expect(')'))
        return false;
      for (int q = 0; q < 3; ++q) {
        if (d[q] < -kMaxApplyRadius || d[q] > kMaxApplyRadius) return fail("offset beyond three cells");
        radius = std::max(radius, std::abs(d[q]));
      }
      char b[96];
      snprintf(b, sizeof(b), "AT(a%d,%d,%d,%d)", idx, d[0], d[1], d[2]);
      *out = b;
      return true;
    }
    if ((c >= '0' && c <= '9') || c == '.') {
      // digits [. digits] [(e|E) [+|-] digits], at least one digit before
      // the exponent (no hexadecimal or other strtod forms)
      auto digit = [&](size_t q) { return s[q] >= '0' && s[q] <= '9'; };
      size_t q = pos;
      int ndig = 0;
      while (digit(q)) ++q, ++ndig;
      if (s[q] == '.') {
        ++q;
        while (digit(q)) ++q, ++ndig;
      }
      if (ndig == 0) return fail("malformed number");
      if (s[q] == 'e' || s[q] == 'E') {
        size_t e = q + 1;
        if (s[e] == '+' || s[e] == '-') ++e;
        if (digit(e)) {
          q = e;
          while (digit(q)) ++q;
        }
      }
      const std::string lit(s + pos, q - pos);
      pos = q;
      const double v = strtod(lit.c_str(), nullptr);
      if (!(v - v == 0.0)) return fail("number out of range");
      char b[64];
      snprintf(b, sizeof(b), "%.17g", v);  // round-trips to the same binary64 value
      *out = std::string("(") + b + ")";
      return true;
    }
    return fail("expected a number, an input reference or '('");
  }
  bool unary(std::string* out) {
    skip();
    if (s[pos] == '-') {
      ++pos;
      if (++depth > kExprMaxDepth) return fail("expression nested too deeply");
      std::string x;
      if (!unary(&x)) return false;
      --depth;
      *out = "(-" + x + ")";
      return true;
    }
    return primary(out);
  }
  bool term(std::string* out) {
    if (!unary(out)) return false;
    for (;;) {
      skip();
      const char c = s[pos];
      if (c != '*' && c != '/') return true;
      ++pos;
      std::string r;
      if (!unary(&r)) return false;
      *out = std::string(c == '*' ? "__dmul_rn(" : "__ddiv_rn(") + *out + ", " + r + ")";
    }
  }
  bool expr(std::string* out) {
    if (++depth > kExprMaxDepth) return fail("expression nested too deeply");
    if (!term(out)) return false;
    for (;;) {
      skip();
      const char c = s[pos];
      if (c != '+' && c != '-') break;
      ++pos;
      std::string r;
      if (!term(&r)) return false;
      *out = std::string(c == '+' ? "__dadd_rn(" : "__dsub_rn(") + *out + ", " + r + ")";
    }
    --depth;
    return true;
  }
};

}  // namespace

// Translates `expr` into the generated kernel's source; *radius receives the
// largest offset (at least 1).
int expr_source(const char* expr, int ninputs, std::string* src, int* radius) {
  if (!expr) return set_error(STENCIL_ERR_ARG, "apply_expr: null expression");
  if (ninputs < 1 || ninputs > kExprMaxInputs)
    return set_error(STENCIL_ERR_ARG, "apply_expr: %d inputs (1..%d)", ninputs, kExprMaxInputs);
  if (strlen(expr) > kExprMaxLen) return set_error(STENCIL_ERR_ARG, "apply_expr: expression longer than 64 KiB");
  ExprParser p{expr, 0, ninputs};
  std::string body;
  if (!p.expr(&body)) return set_error(STENCIL_ERR_ARG, "%s", p.err.c_str());
  p.skip();
  if (expr[p.pos] != '\0') {
    p.fail("unexpected character");
    return set_error(STENCIL_ERR_ARG, "%s", p.err.c_str());
  }
  *radius = std::max(1, p.radius);
  std::string k;
  k += "// generated by stencil_apply_expr\n";
  k += "#define AT(p, dx, dy, dz) (p)[c + (dx) + (long long)(dy) * sy + (long long)(dz) * sz]\n";
  k += "extern \"C\" __global__ void __launch_bounds__(256) stencil_expr_kernel(\n";
  for (int q = 0; q < kExprMaxInputs; ++q) k += "    const double* __restrict__ a" + std::to_string(q) + ",\n";
  k += "    double* __restrict__ out, long long nx, long long ny, long long nz, long long sy, long long sz,\n";
  k += "    long long osy, long long osz, int r) {\n";
  k += "  const long long i = r + (long long)blockIdx.x * 32 + threadIdx.x;\n";
  k += "  const long long j = r + (long long)blockIdx.y * 8 + threadIdx.y;\n";
  k += "  if (i > nx + 1 - r || j > ny + 1 - r) return;\n";
  k += "  for (long long kk = r + blockIdx.z; kk <= nz + 1 - r; kk += gridDim.z) {\n";
  k += "    const long long c = i + j * sy + kk * sz;\n";
  k += "    out[i + j * osy + kk * osz] = " + body + ";\n";
  k += "  }\n}\n";
  *src = k;
  return STENCIL_OK;
}

namespace {

// NVRTC, loaded on first use.
struct Nvrtc {
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  bool ok = false;
};

const Nvrtc& nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    void* h = nullptr;
    for (const char* name : {"libnvrtc.so.13", "libnvrtc.so"})
      if ((h = dlopen(name, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!h) return;
    n.create = reinterpret_cast<decltype(n.create)>(dlsym(h, "nvrtcCreateProgram"));
    n.compile = reinterpret_cast<decltype(n.compile)>(dlsym(h, "nvrtcCompileProgram"));
    n.log_size = reinterpret_cast<decltype(n.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
    n.log = reinterpret_cast<decltype(n.log)>(dlsym(h, "nvrtcGetProgramLog"));
    n.cubin_size = reinterpret_cast<decltype(n.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
    n.cubin = reinterpret_cast<decltype(n.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
    n.destroy = reinterpret_cast<decltype(n.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
    n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy;
  });
  return n;
}

struct ExprKernel {
  cudaLibrary_t lib;
  cudaKernel_t kern;
};

}  // namespace

// Generated kernels of a context, keyed by their source.
struct ExprCache {
  std::mutex mu;
  std::unordered_map<std::string, ExprKernel> m;
};

void expr_cache_free(stencil_ctx* ctx) {
  if (!ctx->expr_cache) return;
  for (auto& kv : ctx->expr_cache->m) cudaLibraryUnload(kv.second.lib);
  delete ctx->expr_cache;
  ctx->expr_cache = nullptr;
}

namespace {

// The compiled kernel for `src` on the ctx's device (compiled and loaded on
// first use).
int expr_kernel(stencil_ctx* ctx, const std::string& src, cudaKernel_t* out) {
  if (!ctx->expr_cache) ctx->expr_cache = new (std::nothrow) ExprCache();
  if (!ctx->expr_cache) return set_error(STENCIL_ERR_ARG, "apply_expr: out of host memory");
  std::lock_guard<std::mutex> lock(ctx->expr_cache->mu);
  auto it = ctx->expr_cache->m.find(src);
  if (it != ctx->expr_cache->m.end()) {
    *out = it->second.kern;
    return STENCIL_OK;
  }
  const Nvrtc& nv = nvrtc();
  if (!nv.ok) return set_error(STENCIL_ERR_CUDA, "apply_expr: the run-time compiler (libnvrtc) is not available");
  cudaDeviceProp prop;
  int rc = check_cuda(cudaGetDeviceProperties(&prop, ctx->device), "cudaGetDeviceProperties");
  if (rc) return rc;
  char arch[48];
  snprintf(arch, sizeof(arch), "--gpu-architecture=sm_%d%da", prop.major, prop.minor);
  const char* opts[] = {arch, "--fmad=false", "-default-device"};
  nvrtcProgram prog;
  if (nv.create(&prog, src.c_str(), "stencil_expr.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
    return set_error(STENCIL_ERR_CUDA, "apply_expr: nvrtcCreateProgram failed");
  const nvrtcResult cr = nv.compile(prog, 3, opts);
  if (cr != NVRTC_SUCCESS) {
    size_t n = 0;
    nv.log_size(prog, &n);
    std::string log(n, '\0');
    if (n) nv.log(prog, &log[0]);
    nv.destroy(&prog);
    return set_error(STENCIL_ERR_CUDA, "apply_expr: compilation failed: %.400s", log.c_str());
  }
  size_t n = 0;
  nv.cubin_size(prog, &n);
  std::vector<char> cubin(n);
  nv.cubin(prog, cubin.data());
  nv.destroy(&prog);
  ExprKernel k;
  rc = check_cuda(cudaLibraryLoadData(&k.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0),
                  "apply_expr: cudaLibraryLoadData");
  if (rc) return rc;
  rc = check_cuda(cudaLibraryGetKernel(&k.kern, k.lib, "stencil_expr_kernel"), "apply_expr: cudaLibraryGetKernel");
  if (rc) {
    cudaLibraryUnload(k.lib);
    return rc;
  }
  ctx->expr_cache->m.emplace(src, k);
  *out = k.kern;
  return STENCIL_OK;
}

}  // namespace

int launch_apply_expr(stencil_ctx* ctx, const Grid* in, int ninputs, const Grid& out, const char* expr,
                      cudaStream_t st) {
  std::string src;
  int r = 1;
  int rc = expr_source(expr, ninputs, &src, &r);
  if (rc) return rc;
  for (int q = 1; q < ninputs; ++q)
    if (in[q].sy != in[0].sy || in[q].sz != in[0].sz)
      return set_error(STENCIL_ERR_ARG, "apply_expr: the inputs must share strides");
  const int64_t ox = in[0].nx + 2 - 2 * r, oy = in[0].ny + 2 - 2 * r, oz = in[0].nz + 2 - 2 * r;
  if (ox < 1 || oy < 1 || oz < 1) return STENCIL_OK;  // nothing to write
  const int64_t gy = (oy + 7) / 8;
  if (gy > 65535) return set_error(STENCIL_ERR_ARG, "apply_expr: ny too large");
  cudaKernel_t kern;
  rc = expr_kernel(ctx, src, &kern);
  if (rc) return rc;
  const double* a[kExprMaxInputs];
  for (int q = 0; q < kExprMaxInputs; ++q) a[q] = static_cast<const double*>(in[q < ninputs ? q : 0].data);
  double* o = static_cast<double*>(out.data);
  long long nx = in[0].nx, ny = in[0].ny, nz = in[0].nz, sy = in[0].sy, sz = in[0].sz, osy = out.sy, osz = out.sz;
  int rr = r;
  void* args[] = {&a[0], &a[1], &a[2], &a[3], &a[4], &a[5], &a[6], &a[7], &o,
                  &nx,   &ny,   &nz,   &sy,   &sz,   &osy,  &osz,  &rr};
  const dim3 grid(static_cast<unsigned>((ox + 31) / 32), static_cast<unsigned>(gy),
                  static_cast<unsigned>(std::min<int64_t>(oz, 65535)));
  return check_cuda(cudaLaunchKernel(reinterpret_cast<const void*>(kern), grid, dim3(32, 8), args, 0, st),
                    "apply_expr launch");
}

}  // namespace stencil
