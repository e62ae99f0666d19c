// srcfuse.cu -- the source-level front-end: Algorithm 1 (Sec. 3.1) applied
// to CUDA source text, compiled at run time with NVRTC.
//
// The paper's tool rewrites two kernels' ASTs with Clang (Sec. 3.3).  Here a
// token-level rewriter does the same for 1-D kernels:
//   * each kernel becomes a __device__ __forceinline__ body that receives its
//     interval context -- thread index tid_k, interval size d_k, barrier id
//     and its dynamic shared-memory slice -- as extra parameters;
//   * in its body threadIdx.x -> tid_k, blockDim.x -> d_k, __syncthreads() ->
//     "bar.sync id_k, d_k", and "extern __shared__ T name[]" -> a pointer to
//     the kernel's slice of the combined dynamic shared memory;
//   * a generated __global__ kernel takes both parameter lists (renamed),
//     sends threads [0, split) to the first body and [split, d0) to the
//     second (the warp-uniform branch of Algorithm 1).
// blockIdx and gridDim pass through unchanged.  Rejected (HF_ERR_UNSUPPORTED):
// threadIdx/blockDim .y/.z, the counting barrier variants, kernel
// templates, file-scope extern __shared__ arrays, block-level builtins
// used outside a kernel body (in a __device__ helper the rewriter would
// have to thread the context through) and in preprocessor lines (a macro
// would carry them into the fused kernel unrewritten).
//
// NVRTC is loaded on first use (dlopen), and the module-loading / launch
// calls of the driver API are resolved through the runtime's driver entry
// point query, so the library has no link-time dependency on either.
#include <cuda.h>
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/hfuse.h"

namespace hf {
hf_status set_last_error(hf_status s, const char *msg);   // runtime.cu
}

namespace {

hf_status err(hf_status s, const std::string &m) { return hf::set_last_error(s, m.c_str()); }

// ------------------------------------------------------------------ lexer
struct Tok {
    enum Kind { Ident, Number, String, Char, Punct, PP } kind;
    std::string text;
    std::string pre;   // whitespace and comments before the token
};

bool is_id0(char c) { return (c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z') || c == '_'; }
bool is_id(char c) { return is_id0(c) || (c >= '0' && c <= '9'); }
bool is_digit(char c) { return c >= '0' && c <= '9'; }

bool lex(const std::string &s, std::vector<Tok> &out, std::string &why)
{
    size_t i = 0, n = s.size();
    bool line_start = true;
    std::string pre;
    while (i < n) {
        const char c = s[i];
        if (c == ' ' || c == '\t' || c == '\r' || c == '\n' || c == '\f' || c == '\v') {
            if (c == '\n') line_start = true;
            pre += c;
            ++i;
            continue;
        }
        if (c == '/' && i + 1 < n && s[i + 1] == '/') {
            while (i < n && s[i] != '\n') pre += s[i++];
            continue;
        }
        if (c == '/' && i + 1 < n && s[i + 1] == '*') {
            const size_t e = s.find("*/", i + 2);
            if (e == std::string::npos) {
                why = "unterminated comment";
                return false;
            }
            pre += s.substr(i, e + 2 - i);
            i = e + 2;
            continue;
        }
        Tok t;
        t.pre.swap(pre);
        const size_t b = i;
        if (c == '#' && line_start) {
            // a preprocessor line, with backslash continuations
            while (i < n && s[i] != '\n') {
                if (s[i] == '\\' && i + 1 < n && s[i + 1] == '\n') i += 2;
                else ++i;
            }
            t.kind = Tok::PP;
        } else if (is_id0(c)) {
            while (i < n && is_id(s[i])) ++i;
            t.kind = Tok::Ident;
        } else if (is_digit(c) || (c == '.' && i + 1 < n && is_digit(s[i + 1]))) {
            while (i < n && (is_id(s[i]) || s[i] == '.' ||
                             ((s[i] == '+' || s[i] == '-') &&
                              (s[i - 1] == 'e' || s[i - 1] == 'E' || s[i - 1] == 'p' || s[i - 1] == 'P'))))
                ++i;
            t.kind = Tok::Number;
        } else if (c == '"' || c == '\'') {
            ++i;
            while (i < n && s[i] != c) {
                if (s[i] == '\\') ++i;
                if (i < n && s[i] == '\n') break;
                ++i;
            }
            if (i >= n || s[i] != c) {
                why = "unterminated literal";
                return false;
            }
            ++i;
            t.kind = c == '"' ? Tok::String : Tok::Char;
        } else {
            t.kind = Tok::Punct;
            if (i + 1 < n && ((c == '-' && s[i + 1] == '>') || (c == ':' && s[i + 1] == ':'))) i += 2;
            else ++i;
        }
        t.text = s.substr(b, i - b);
        line_start = false;
        out.push_back(std::move(t));
    }
    if (!pre.empty()) out.push_back(Tok{Tok::Punct, "", pre});   // trailing trivia
    return true;
}

bool is(const std::vector<Tok> &t, size_t i, const char *s)
{
    return i < t.size() && t[i].text == s;
}

// index of the token closing the bracket opened at `open`, or npos
size_t match(const std::vector<Tok> &t, size_t open)
{
    const std::string o = t[open].text;
    const std::string c = o == "(" ? ")" : o == "{" ? "}" : o == "[" ? "]" : "";
    int depth = 0;
    for (size_t i = open; i < t.size(); ++i) {
        if (t[i].kind != Tok::Punct) continue;
        if (t[i].text == o) ++depth;
        else if (t[i].text == c && --depth == 0) return i;
    }
    return std::string::npos;
}

// ------------------------------------------------------------------ kernels
struct Param {
    size_t b, e;         // token range [b, e)
    size_t name;         // token index of the parameter's name
};

struct Kernel {
    std::string name;
    size_t head;         // first token of the signature to replace (extern / __global__)
    size_t lparen, rparen, lbrace, rbrace;
    std::vector<Param> params;
};

// Every __global__ function definition of the token stream.
bool find_kernels(const std::vector<Tok> &t, std::vector<Kernel> &ks, std::string &why)
{
    for (size_t g = 0; g < t.size(); ++g) {
        if (!(t[g].kind == Tok::Ident && t[g].text == "__global__")) continue;
        Kernel k;
        k.head = g;
        if (g >= 2 && is(t, g - 2, "extern") && t[g - 1].kind == Tok::String) k.head = g - 2;
        size_t h = k.head;
        if (h >= 1 && is(t, h - 1, ">")) {
            why = "kernel templates are not supported (instantiate the kernel first)";
            return false;
        }
        // walk to the parameter list, skipping __launch_bounds__(...) and the like
        size_t i = g + 1, name = std::string::npos;
        while (i < t.size()) {
            if (t[i].kind == Tok::Punct && t[i].text == "(") {
                if (name != std::string::npos && i == name + 1 &&
                    t[name].text.compare(0, 2, "__") != 0)
                    break;
                const size_t m = match(t, i);
                if (m == std::string::npos) {
                    why = "unbalanced parentheses";
                    return false;
                }
                i = m + 1;
                continue;
            }
            if (t[i].kind == Tok::Ident) name = i;
            else if (t[i].kind == Tok::Punct && (t[i].text == ";" || t[i].text == "{")) break;
            ++i;
        }
        if (i >= t.size() || t[i].text != "(") continue;   // a declaration we cannot read
        k.name = t[name].text;
        k.lparen = i;
        k.rparen = match(t, i);
        if (k.rparen == std::string::npos) {
            why = "unbalanced parentheses";
            return false;
        }
        if (!is(t, k.rparen + 1, "{")) continue;   // a declaration, not a definition
        k.lbrace = k.rparen + 1;
        k.rbrace = match(t, k.lbrace);
        if (k.rbrace == std::string::npos) {
            why = "unbalanced braces in " + k.name;
            return false;
        }
        // parameters: split on top-level commas; the name is the last identifier
        size_t b = k.lparen + 1;
        int depth = 0;
        for (size_t j = k.lparen + 1; j <= k.rparen; ++j) {
            const std::string &x = t[j].text;
            if (t[j].kind == Tok::Punct && (x == "(" || x == "[" || x == "<")) ++depth;
            if (t[j].kind == Tok::Punct && (x == ")" || x == "]" || x == ">") && j != k.rparen) --depth;
            if (j == k.rparen || (depth == 0 && t[j].kind == Tok::Punct && x == ",")) {
                if (j > b && !(j == b + 1 && is(t, b, "void"))) {
                    Param p{b, j, std::string::npos};
                    for (size_t q = b; q < j; ++q)
                        if (t[q].kind == Tok::Ident && t[q].text != "__restrict__" &&
                            t[q].text != "const" && t[q].text != "__grid_constant__")
                            p.name = q;
                    if (p.name == std::string::npos) {
                        why = "unnamed parameter in " + k.name;
                        return false;
                    }
                    k.params.push_back(p);
                }
                b = j + 1;
            }
        }
        ks.push_back(k);
        g = k.rbrace;
    }
    return true;
}

std::string text(const std::vector<Tok> &t, size_t b, size_t e, bool first_pre = true)
{
    std::string s;
    for (size_t i = b; i < e; ++i) {
        if (i > b || first_pre) s += t[i].pre;
        s += t[i].text;
    }
    return s;
}

// Checks a token range outside kernel bodies for block-level builtins.
bool builtin(const std::string &x)
{
    return x == "threadIdx" || x == "blockDim" || x.compare(0, 13, "__syncthreads") == 0;
}

// True when a preprocessor line names a block-level builtin: a macro would
// carry it past the rewriter into the fused kernel unchanged.
bool pp_builtin(const std::string &line)
{
    for (size_t i = 0; i < line.size();) {
        if (is_id0(line[i])) {
            const size_t b = i;
            while (i < line.size() && is_id(line[i])) ++i;
            if (builtin(line.substr(b, i - b))) return true;
        } else {
            ++i;
        }
    }
    return false;
}

// Rewrites one kernel into an interval body; appends the new text of tokens
// [k.head, k.rbrace] to `out`.
bool rewrite_kernel(const std::vector<Tok> &t, const Kernel &k, std::string &out, std::string &why)
{
    out += t[k.head].pre;
    out += "__device__ __forceinline__ void " + k.name + "__hf_body(";
    for (size_t p = 0; p < k.params.size(); ++p) {
        std::string d;
        for (size_t q = k.params[p].b; q < k.params[p].e; ++q) {
            if (t[q].text == "__grid_constant__") continue;   // only valid on kernels
            d += t[q].pre + t[q].text;
        }
        out += d + ", ";
    }
    out += "unsigned hf_tid_, unsigned hf_ntid_, unsigned hf_bar_, unsigned char *hf_dyn_)";
    out += t[k.lbrace].pre + "{";
    for (size_t i = k.lbrace + 1; i < k.rbrace; ++i) {
        const Tok &x = t[i];
        if (x.kind == Tok::Ident && (x.text == "threadIdx" || x.text == "blockDim")) {
            if (!(is(t, i + 1, ".") && t[i + 2].kind == Tok::Ident)) {
                why = x.text + " used as a whole in " + k.name + " (only ." + "x is supported)";
                return false;
            }
            if (t[i + 2].text != "x") {
                why = x.text + "." + t[i + 2].text + " in " + k.name + ": only 1-D blocks are supported";
                return false;
            }
            out += x.pre + (x.text == "threadIdx" ? "hf_tid_" : "hf_ntid_");
            i += 2;
        } else if (x.kind == Tok::Ident && x.text == "__syncthreads") {
            if (!(is(t, i + 1, "(") && is(t, i + 2, ")"))) {
                why = "malformed __syncthreads() in " + k.name;
                return false;
            }
            out += x.pre + "hf_bar_sync_(hf_bar_, hf_ntid_)";
            i += 2;
        } else if (x.kind == Tok::Ident && x.text.compare(0, 14, "__syncthreads_") == 0) {
            why = x.text + " in " + k.name + " is not supported";
            return false;
        } else if (x.kind == Tok::Ident && x.text == "extern" && is(t, i + 1, "__shared__")) {
            // extern __shared__ [__align__(n)] T name[];  ->  T *name = (T *)hf_dyn_;
            size_t j = i + 2, lb = std::string::npos;
            std::string type;
            while (j < k.rbrace && !is(t, j, ";")) {
                if (is(t, j, "__align__") && is(t, j + 1, "(")) {
                    j = match(t, j + 1) + 1;
                    continue;
                }
                if (is(t, j, "[")) {
                    lb = j;
                    break;
                }
                type += (type.empty() ? "" : " ") + t[j].text;
                ++j;
            }
            const size_t nm = lb == std::string::npos ? lb : lb - 1;
            if (lb == std::string::npos || t[nm].kind != Tok::Ident || !is(t, lb + 1, "]") ||
                !is(t, lb + 2, ";")) {
                why = "unsupported extern __shared__ declaration in " + k.name;
                return false;
            }
            type = type.substr(0, type.size() - t[nm].text.size());
            while (!type.empty() && type.back() == ' ') type.pop_back();
            out += x.pre + type + " *" + t[nm].text + " = reinterpret_cast<" + type + " *>(hf_dyn_);";
            i = lb + 2;
        } else {
            out += x.pre + x.text;
        }
    }
    out += t[k.rbrace].pre + "}";
    return true;
}

// Rewrites `src` so that kernels named in `names` become interval bodies.
bool rewrite_source(const std::string &src, const std::vector<std::string> &names,
                    std::string &out, std::vector<Kernel> &found, std::string &why, hf_status &code)
{
    std::vector<Tok> t;
    code = HF_ERR_INVALID;
    if (!lex(src, t, why)) return false;
    std::vector<Kernel> ks;
    code = HF_ERR_UNSUPPORTED;
    if (!find_kernels(t, ks, why)) return false;
    // builtins outside every kernel body
    for (size_t i = 0; i < t.size(); ++i) {
        bool inside = false;
        for (const Kernel &k : ks)
            if (i > k.lbrace && i < k.rbrace) inside = true;
        if (!inside && t[i].kind == Tok::Ident && builtin(t[i].text)) {
            why = t[i].text + " outside a kernel body (a __device__ helper): inline it into the kernel";
            return false;
        }
        if (t[i].kind == Tok::PP && pp_builtin(t[i].text)) {
            why = "a preprocessor line names threadIdx, blockDim or __syncthreads (a macro is not "
                  "rewritten): expand it in the kernel";
            return false;
        }
        if (!inside && is(t, i, "extern") && is(t, i + 1, "__shared__")) {
            why = "file-scope extern __shared__ arrays are not supported: declare them in the kernel";
            return false;
        }
    }
    found.clear();
    for (const std::string &n : names) {
        const Kernel *hit = nullptr;
        for (const Kernel &k : ks)
            if (k.name == n) {
                if (hit) {
                    code = HF_ERR_INVALID;
                    why = "kernel " + n + " is defined twice";
                    return false;
                }
                hit = &k;
            }
        if (!hit) {
            code = HF_ERR_INVALID;
            why = "no __global__ definition named " + n;
            return false;
        }
        bool dup = false;
        for (const Kernel &f : found) dup |= f.name == n;
        if (!dup) found.push_back(*hit);
    }
    size_t pos = 0;
    out.clear();
    std::vector<Kernel> order = found;
    std::sort(order.begin(), order.end(), [](const Kernel &a, const Kernel &b) { return a.head < b.head; });
    for (const Kernel &k : order) {
        out += text(t, pos, k.head);
        if (!rewrite_kernel(t, k, out, why)) return false;
        pos = k.rbrace + 1;
    }
    out += text(t, pos, t.size());
    code = HF_OK;
    return true;
}

std::string param_list(const std::vector<Tok> &t, const Kernel &k, const char *prefix, std::string &call)
{
    std::string decl;
    for (size_t p = 0; p < k.params.size(); ++p) {
        const Param &q = k.params[p];
        const std::string nm = std::string(prefix) + std::to_string(p);
        for (size_t j = q.b; j < q.e; ++j) {
            decl += (j == q.b ? std::string(" ") : t[j].pre);
            decl += j == q.name ? nm : t[j].text;
        }
        decl += ",";
        call += nm + ", ";
    }
    return decl;
}

// The fused source of Algorithm 1 for kernels a (threads [0, split)) and b.
hf_status fuse_source(const char *src_a, const char *name_a, const char *src_b, const char *name_b,
                      int split, int d0, std::string &out)
{
    if (!src_a || !name_a || !name_b) return err(HF_ERR_INVALID, "NULL source or kernel name");
    if (d0 <= 0 || d0 > 1024 || d0 % 32 || split <= 0 || split >= d0 || split % 32)
        return err(HF_ERR_SPLIT, "split " + std::to_string(split) + " of " + std::to_string(d0) +
                                     ": need multiples of 32 with 0 < split < d0 <= 1024");
    const bool same = !src_b || std::strcmp(src_a, src_b) == 0;
    std::string ra, rb, why;
    std::vector<Kernel> ka, kb;
    hf_status code;
    std::vector<Tok> ta, tb;
    std::string w;
    lex(src_a, ta, w);
    if (same) {
        if (!rewrite_source(src_a, {name_a, name_b}, ra, ka, why, code)) return err(code, why);
    } else {
        lex(src_b, tb, w);
        if (!rewrite_source(src_a, {name_a}, ra, ka, why, code)) return err(code, why);
        if (!rewrite_source(src_b, {name_b}, rb, kb, why, code)) return err(code, why);
    }
    // token streams for the parameter declarations
    std::vector<Kernel> all_a, all_b;
    find_kernels(ta, all_a, w);
    if (!same) find_kernels(tb, all_b, w);
    const std::vector<Tok> &tB = same ? ta : tb;
    const std::vector<Kernel> &kB = same ? all_a : all_b;
    const Kernel *A = nullptr, *B = nullptr;
    for (const Kernel &k : all_a)
        if (k.name == name_a) A = &k;
    for (const Kernel &k : kB)
        if (k.name == name_b) B = &k;
    if (!A || !B) return err(HF_ERR_INVALID, "kernel not found");
    std::string call_a, call_b;
    const std::string pa = param_list(ta, *A, "hf_a", call_a);
    const std::string pb = param_list(tB, *B, "hf_b", call_b);
    const std::string s = std::to_string(split) + "u", d = std::to_string(d0 - split) + "u";
    out = "// Horizontally fused by hf_src_fuse (Algorithm 1): " + std::string(name_a) + " on threads [0, " +
          std::to_string(split) + "), " + name_b + " on [" + std::to_string(split) + ", " +
          std::to_string(d0) + ").\n"
          "__device__ __forceinline__ void hf_bar_sync_(unsigned id, unsigned n)\n"
          "{\n    asm volatile(\"bar.sync %0, %1;\" ::\"r\"(id), \"r\"(n) : \"memory\");\n}\n"
          "#line 1 \"kernel_a\"\n" + ra + "\n";
    if (!same) out += "#line 1 \"kernel_b\"\n" + rb + "\n";
    out += "extern \"C\" __global__ void __launch_bounds__(" + std::to_string(d0) + ") hf_src_fused(" + pa +
           pb + " unsigned hf_dyn_off_)\n{\n"
           "    extern __shared__ __align__(128) unsigned char hf_dyn_smem_[];\n"
           "    if (threadIdx.x < " + s + ")\n        " + std::string(name_a) + "__hf_body(" + call_a +
           "threadIdx.x, " + s + ", 1u, hf_dyn_smem_);\n"
           "    else\n        " + std::string(name_b) + "__hf_body(" + call_b + "threadIdx.x - " + s + ", " +
           d + ", 2u, hf_dyn_smem_ + hf_dyn_off_);\n}\n";
    return HF_OK;
}

// ------------------------------------------------------------------ NVRTC
struct Nvrtc {
    bool ok = false;
    std::string why;
    nvrtcResult (*create)(nvrtcProgram *, const char *, const char *, int, const char *const *,
                          const char *const *);
    nvrtcResult (*compile)(nvrtcProgram, int, const char *const *);
    nvrtcResult (*log_size)(nvrtcProgram, size_t *);
    nvrtcResult (*log)(nvrtcProgram, char *);
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t *);
    nvrtcResult (*cubin)(nvrtcProgram, char *);
    nvrtcResult (*add_name)(nvrtcProgram, const char *);
    nvrtcResult (*lowered)(nvrtcProgram, const char *, const char **);
    nvrtcResult (*destroy)(nvrtcProgram *);
};

const Nvrtc &nvrtc()
{
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        // found through the library's run path (the CUDA library directory)
        void *h = nullptr;
        for (const char *name : {"libnvrtc.so.13", "libnvrtc.so"}) {
            h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
            if (h) break;
        }
        if (!h) {
            n.why = "NVRTC (libnvrtc.so) could not be loaded";
            return;
        }
        bool all = true;
        auto get = [&](auto &fp, const char *sym) {
            void *p = dlsym(h, sym);
            all &= p != nullptr;
            fp = reinterpret_cast<std::remove_reference_t<decltype(fp)>>(p);
        };
        get(n.create, "nvrtcCreateProgram");
        get(n.compile, "nvrtcCompileProgram");
        get(n.log_size, "nvrtcGetProgramLogSize");
        get(n.log, "nvrtcGetProgramLog");
        get(n.cubin_size, "nvrtcGetCUBINSize");
        get(n.cubin, "nvrtcGetCUBIN");
        get(n.add_name, "nvrtcAddNameExpression");
        get(n.lowered, "nvrtcGetLoweredName");
        get(n.destroy, "nvrtcDestroyProgram");
        n.ok = all;
        if (!all) n.why = "NVRTC is missing an entry point";
    });
    return n;
}

std::string arch_option()
{
    int dev = 0, major = 10, minor = 3;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    }
    cudaGetLastError();   // no device here is not an error for a compile
    return "--gpu-architecture=sm_" + std::to_string(major) + std::to_string(minor) + "a";
}

// Compiles `src`; on success returns the cubin and the lowered name of `name`.
hf_status compile(const std::string &src, const char *name, int regcap, std::vector<char> &cubin,
                  std::string &lowered, std::string *log_out)
{
    const Nvrtc &N = nvrtc();
    if (!N.ok) return err(HF_ERR_UNSUPPORTED, N.why);
    if (regcap != 0 && (regcap < 24 || regcap > 255)) return err(HF_ERR_INVALID, "regcap out of range");
    nvrtcProgram prog;
    if (N.create(&prog, src.c_str(), "hf_src.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
        return err(HF_ERR_INVALID, "nvrtcCreateProgram failed");
    const std::string arch = arch_option(), cap = "--maxrregcount=" + std::to_string(regcap);
    std::vector<const char *> opts = {arch.c_str(), "-std=c++17", "-lineinfo"};
    if (regcap) opts.push_back(cap.c_str());
    const std::string expr = std::string("&") + name;
    N.add_name(prog, expr.c_str());
    const nvrtcResult r = N.compile(prog, (int)opts.size(), opts.data());
    size_t ls = 0;
    N.log_size(prog, &ls);
    std::string log(ls, '\0');
    if (ls) N.log(prog, &log[0]);
    if (log_out) *log_out = log;
    if (r != NVRTC_SUCCESS) {
        N.destroy(&prog);
        return err(HF_ERR_INVALID, "NVRTC compile failed: " + log.substr(0, 400));
    }
    const char *low = nullptr;
    if (N.lowered(prog, expr.c_str(), &low) != NVRTC_SUCCESS || !low) {
        N.destroy(&prog);
        return err(HF_ERR_INVALID, std::string("no kernel named ") + name + " in the compiled source");
    }
    lowered = low;
    size_t cs = 0;
    N.cubin_size(prog, &cs);
    cubin.resize(cs);
    N.cubin(prog, cubin.data());
    N.destroy(&prog);
    return HF_OK;
}

// ------------------------------------------------------------------ driver API
struct Driver {
    bool ok = false;
    CUresult (*load)(CUmodule *, const void *);
    CUresult (*get)(CUfunction *, CUmodule, const char *);
    CUresult (*unload)(CUmodule);
    CUresult (*launch)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                       CUstream, void **, void **);
    CUresult (*attr)(int *, CUfunction_attribute, CUfunction);
    CUresult (*set_attr)(CUfunction, CUfunction_attribute, int);
};

const Driver &driver()
{
    static Driver d;
    static std::once_flag once;
    std::call_once(once, [] {
        bool all = true;
        auto get = [&](auto &fp, const char *sym) {
            void *p = nullptr;
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion(sym, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
                q != cudaDriverEntryPointSuccess)
                p = nullptr;
            all &= p != nullptr;
            fp = reinterpret_cast<std::remove_reference_t<decltype(fp)>>(p);
        };
        get(d.load, "cuModuleLoadData");
        get(d.get, "cuModuleGetFunction");
        get(d.unload, "cuModuleUnload");
        get(d.launch, "cuLaunchKernel");
        get(d.attr, "cuFuncGetAttribute");
        get(d.set_attr, "cuFuncSetAttribute");
        cudaGetLastError();
        d.ok = all;
    });
    return d;
}

} // namespace

struct hf_src_module_t {
    CUmodule mod = nullptr;
    CUfunction fn = nullptr;
    int fused = 0;
    int n_a = 0, n_b = 0;   // parameters of each constituent (fused modules)
    int d0 = 0;
    std::string source;
};

extern "C" {

hf_status hf_src_fuse(const char *src_a, const char *name_a, const char *src_b, const char *name_b,
                      int split, int d0, char *out, size_t cap, size_t *len)
{
    std::string s;
    hf_status st = fuse_source(src_a, name_a, src_b, name_b, split, d0, s);
    if (st) return st;
    if (len) *len = s.size() + 1;
    if (out && cap) {
        const size_t n = std::min(cap - 1, s.size());
        std::memcpy(out, s.data(), n);
        out[n] = '\0';
        if (n < s.size()) return err(HF_ERR_INVALID, "output buffer too small");
    }
    return HF_OK;
}

hf_status hf_src_compile_check(const char *src, const char *name, int regcap, char *log, size_t cap)
{
    if (!src || !name) return err(HF_ERR_INVALID, "NULL source or kernel name");
    std::vector<char> cubin;
    std::string lowered, lg;
    hf_status st = compile(src, name, regcap, cubin, lowered, &lg);
    if (log && cap) {
        const size_t n = std::min(cap - 1, lg.size());
        std::memcpy(log, lg.data(), n);
        log[n] = '\0';
    }
    return st;
}

static hf_status load(const std::string &src, const char *name, int regcap, hf_src_module_t *m)
{
    std::vector<char> cubin;
    std::string lowered;
    hf_status st = compile(src, name, regcap, cubin, lowered, nullptr);
    if (st) return st;
    const Driver &D = driver();
    if (!D.ok) return err(HF_ERR_CUDA, "driver entry points unavailable");
    cudaFree(nullptr);   // make the primary context current
    if (D.load(&m->mod, cubin.data()) != CUDA_SUCCESS) return err(HF_ERR_CUDA, "cuModuleLoadData failed");
    if (D.get(&m->fn, m->mod, lowered.c_str()) != CUDA_SUCCESS) {
        D.unload(m->mod);
        return err(HF_ERR_CUDA, "cuModuleGetFunction failed");
    }
    m->source = src;
    return HF_OK;
}

hf_status hf_src_load(const char *src, const char *name, int regcap, hf_src_module *out)
{
    if (!src || !name || !out) return err(HF_ERR_INVALID, "NULL argument");
    auto *m = new hf_src_module_t;
    hf_status st = load(src, name, regcap, m);
    if (st) {
        delete m;
        return st;
    }
    *out = m;
    return HF_OK;
}

hf_status hf_src_fuse_load(const char *src_a, const char *name_a, const char *src_b, const char *name_b,
                           int split, int d0, int regcap, hf_src_module *out)
{
    if (!out) return err(HF_ERR_INVALID, "NULL output");
    std::string s;
    hf_status st = fuse_source(src_a, name_a, src_b, name_b, split, d0, s);
    if (st) return st;
    // parameter counts, for the launch
    std::vector<Tok> ta, tb;
    std::vector<Kernel> ka, kb;
    std::string w;
    lex(src_a, ta, w);
    find_kernels(ta, ka, w);
    lex(src_b ? src_b : src_a, tb, w);
    find_kernels(tb, kb, w);
    auto *m = new hf_src_module_t;
    for (const Kernel &k : ka)
        if (k.name == name_a) m->n_a = (int)k.params.size();
    for (const Kernel &k : kb)
        if (k.name == name_b) m->n_b = (int)k.params.size();
    m->fused = 1;
    m->d0 = d0;
    st = load(s, "hf_src_fused", regcap, m);
    if (st) {
        delete m;
        return st;
    }
    *out = m;
    return HF_OK;
}

static hf_status launch(hf_src_module m, void **params, int grid, int block, size_t smem, void *stream)
{
    const Driver &D = driver();
    if (!D.ok) return err(HF_ERR_CUDA, "driver entry points unavailable");
    int maxthr = 0;
    D.attr(&maxthr, CU_FUNC_ATTRIBUTE_MAX_THREADS_PER_BLOCK, m->fn);
    if (block <= 0 || block > maxthr)
        return err(HF_ERR_REGS, "block of " + std::to_string(block) + " threads: the kernel allows " +
                                    std::to_string(maxthr));
    if (grid <= 0) return err(HF_ERR_INVALID, "grid must be positive");
    if (smem > 48 * 1024) {
        int optin = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        int stat = 0;
        D.attr(&stat, CU_FUNC_ATTRIBUTE_SHARED_SIZE_BYTES, m->fn);
        if ((long)smem + stat > optin) return err(HF_ERR_SMEM, "dynamic shared memory over the per-block limit");
        if (D.set_attr(m->fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)smem) != CUDA_SUCCESS)
            return err(HF_ERR_CUDA, "cuFuncSetAttribute failed");
    }
    if (D.launch(m->fn, (unsigned)grid, 1, 1, (unsigned)block, 1, 1, (unsigned)smem,
                 static_cast<CUstream>(stream), params, nullptr) != CUDA_SUCCESS)
        return err(HF_ERR_CUDA, "cuLaunchKernel failed");
    return HF_OK;
}

hf_status hf_src_launch(hf_src_module m, void **params, int grid, int block, size_t dyn_smem, void *stream)
{
    if (!m || m->fused) return err(HF_ERR_INVALID, "not a single-kernel module");
    return launch(m, params, grid, block, dyn_smem, stream);
}

hf_status hf_src_launch_fused(hf_src_module m, void **params_a, void **params_b, size_t dyn_smem_a,
                              size_t dyn_smem_b, int grid, void *stream)
{
    if (!m || !m->fused) return err(HF_ERR_INVALID, "not a fused module");
    if ((m->n_a && !params_a) || (m->n_b && !params_b)) return err(HF_ERR_INVALID, "NULL parameter array");
    const size_t off = (dyn_smem_a + 127) / 128 * 128;
    unsigned off32 = (unsigned)off;
    std::vector<void *> p;
    for (int i = 0; i < m->n_a; ++i) p.push_back(params_a[i]);
    for (int i = 0; i < m->n_b; ++i) p.push_back(params_b[i]);
    p.push_back(&off32);
    return launch(m, p.data(), grid, m->d0, off + dyn_smem_b, stream);
}

hf_status hf_src_query(hf_src_module m, int *regs, int *local_bytes, int *static_smem, int *max_threads)
{
    if (!m) return err(HF_ERR_INVALID, "NULL module");
    const Driver &D = driver();
    if (!D.ok) return err(HF_ERR_CUDA, "driver entry points unavailable");
    if (regs) D.attr(regs, CU_FUNC_ATTRIBUTE_NUM_REGS, m->fn);
    if (local_bytes) D.attr(local_bytes, CU_FUNC_ATTRIBUTE_LOCAL_SIZE_BYTES, m->fn);
    if (static_smem) D.attr(static_smem, CU_FUNC_ATTRIBUTE_SHARED_SIZE_BYTES, m->fn);
    if (max_threads) D.attr(max_threads, CU_FUNC_ATTRIBUTE_MAX_THREADS_PER_BLOCK, m->fn);
    return HF_OK;
}

void hf_src_unload(hf_src_module m)
{
    if (!m) return;
    if (m->mod && driver().ok) driver().unload(m->mod);
    delete m;
}

} // extern "C"
