// checkpoint.cu -- checkpoints of a trained drag closure (host code only).
//
// A checkpoint is two files beside each other:
//   <path>.f32   the CG_MLP_NPARAM parameters as little-endian float32 in the
//                ABI order (W1, b1, W2, b2, w3, b3);
//   <path>.json  a JSON object: "format": "dual-grid drag closure",
//                "version": 1, the network sizes ("nparam", "nfeat",
//                "hidden", "k0"), "params_file" (the .f32 file's name),
//                "params_sha256" (SHA-256 of the .f32 file, lower-case hex),
//                "feature_lo" / "feature_hi" (the feature box, floats written
//                as the doubles they are), "activation" ("gelu" or "relu";
//                absent: "gelu") and "meta" (any JSON object).
// Python's closure.save_checkpoint / load_checkpoint read and write the same
// files.  SHA-256 follows FIPS 180-4; its round constants and initial hash
// are formed here from their definition (the fractional parts of the cube
// and square roots of the first primes) with exact integer roots.
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <string>
#include <vector>

#include "cg_internal.cuh"

namespace {

// ---------------------------------------------------------------- SHA-256
typedef unsigned __int128 u128;

// Largest y with y^k <= v (k = 2 or 3), by bisection on integers.
uint64_t iroot(u128 v, int k) {
    uint64_t lo = 0, hi = (uint64_t)1 << 40;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo + 1) / 2;
        u128 p = (u128)mid * mid;
        if (k == 3) p *= mid;
        if (p <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct ShaConst {
    uint32_t k[64], h0[8];
    ShaConst() {
        int found = 0;
        for (uint32_t p = 2; found < 64; ++p) {
            bool prime = true;
            for (uint32_t d = 2; d * d <= p; ++d)
                if (p % d == 0) {
                    prime = false;
                    break;
                }
            if (!prime) continue;
            // first 32 bits of the fractional part of p^(1/3): floor(p^(1/3) 2^32) mod 2^32
            k[found] = (uint32_t)iroot((u128)p << 96, 3);
            // of p^(1/2), for the first eight primes
            if (found < 8) h0[found] = (uint32_t)iroot((u128)p << 64, 2);
            ++found;
        }
    }
};

const ShaConst& sha_const() {
    static const ShaConst c;
    return c;
}

inline uint32_t rotr(uint32_t x, int r) { return (x >> r) | (x << (32 - r)); }

std::string sha256_hex(const unsigned char* data, size_t len) {
    const ShaConst& C = sha_const();
    uint32_t h[8];
    memcpy(h, C.h0, sizeof h);
    // message, a 1 bit, zeros, and the length in bits (big-endian 64-bit)
    std::vector<unsigned char> m(data, data + len);
    m.push_back(0x80);
    while (m.size() % 64 != 56) m.push_back(0);
    const uint64_t bits = (uint64_t)len * 8;
    for (int i = 7; i >= 0; --i) m.push_back((unsigned char)(bits >> (8 * i)));
    for (size_t off = 0; off < m.size(); off += 64) {
        uint32_t w[64];
        for (int t = 0; t < 16; ++t)
            w[t] = (uint32_t)m[off + 4 * t] << 24 | (uint32_t)m[off + 4 * t + 1] << 16 |
                   (uint32_t)m[off + 4 * t + 2] << 8 | (uint32_t)m[off + 4 * t + 3];
        for (int t = 16; t < 64; ++t) {
            const uint32_t s0 = rotr(w[t - 15], 7) ^ rotr(w[t - 15], 18) ^ (w[t - 15] >> 3);
            const uint32_t s1 = rotr(w[t - 2], 17) ^ rotr(w[t - 2], 19) ^ (w[t - 2] >> 10);
            w[t] = w[t - 16] + s0 + w[t - 7] + s1;
        }
        uint32_t a = h[0], b = h[1], c = h[2], d = h[3], e = h[4], f = h[5], g = h[6], hh = h[7];
        for (int t = 0; t < 64; ++t) {
            const uint32_t S1 = rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25);
            const uint32_t ch = (e & f) ^ (~e & g);
            const uint32_t t1 = hh + S1 + ch + C.k[t] + w[t];
            const uint32_t S0 = rotr(a, 2) ^ rotr(a, 13) ^ rotr(a, 22);
            const uint32_t maj = (a & b) ^ (a & c) ^ (b & c);
            const uint32_t t2 = S0 + maj;
            hh = g;
            g = f;
            f = e;
            e = d + t1;
            d = c;
            c = b;
            b = a;
            a = t1 + t2;
        }
        h[0] += a; h[1] += b; h[2] += c; h[3] += d;
        h[4] += e; h[5] += f; h[6] += g; h[7] += hh;
    }
    static const char* hex = "0123456789abcdef";
    std::string out;
    for (int i = 0; i < 8; ++i)
        for (int s = 28; s >= 0; s -= 4) out.push_back(hex[(h[i] >> s) & 15u]);
    return out;
}

// ---------------------------------------------------------------- JSON
// A small reader for the head: the top-level object's members are kept as
// numbers, strings or arrays of numbers; any other value (the meta object)
// is checked for well-formedness and skipped.
struct Json {
    const char* p;
    const char* e;
    bool ok = true;

    void ws() {
        while (p < e && (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t')) ++p;
    }
    bool lit(const char* s) {
        const size_t k = strlen(s);
        if ((size_t)(e - p) >= k && memcmp(p, s, k) == 0) {
            p += k;
            return true;
        }
        return false;
    }
    bool str(std::string* out) {
        ws();
        if (p >= e || *p != '"') return ok = false;
        ++p;
        while (p < e && *p != '"') {
            if (*p == '\\') {
                ++p;
                if (p >= e) return ok = false;
                const char c = *p;
                if (c == 'u') {
                    if (e - p < 5) return ok = false;
                    p += 4;   // kept only for skipping; the head's own strings are ASCII
                    if (out) out->push_back('?');
                } else if (out) {
                    out->push_back(c == 'n' ? '\n' : c == 't' ? '\t' : c == 'r' ? '\r' : c == 'b' ? '\b'
                                                                         : c == 'f' ? '\f' : c);
                }
            } else if (out) {
                out->push_back(*p);
            }
            ++p;
        }
        if (p >= e) return ok = false;
        ++p;
        return true;
    }
    bool num(double* out) {
        ws();
        char buf[64];
        size_t k = 0;
        while (p < e && k < sizeof buf - 1 && (strchr("+-0123456789.eE", *p) != nullptr)) buf[k++] = *p++;
        buf[k] = 0;
        if (!k) return ok = false;
        char* end = nullptr;
        const double v = strtod(buf, &end);
        if (end != buf + k) return ok = false;
        if (out) *out = v;
        return true;
    }
    bool skip(int depth = 0) {   // any value
        ws();
        if (p >= e || depth > 64) return ok = false;
        if (*p == '"') return str(nullptr);
        if (*p == '{' || *p == '[') {
            const char close = *p == '{' ? '}' : ']';
            const bool obj = *p == '{';
            ++p;
            ws();
            if (p < e && *p == close) {
                ++p;
                return true;
            }
            for (;;) {
                if (obj) {
                    if (!str(nullptr)) return false;
                    ws();
                    if (p >= e || *p != ':') return ok = false;
                    ++p;
                }
                if (!skip(depth + 1)) return false;
                ws();
                if (p < e && *p == ',') {
                    ++p;
                    continue;
                }
                if (p < e && *p == close) {
                    ++p;
                    return true;
                }
                return ok = false;
            }
        }
        if (lit("true") || lit("false") || lit("null")) return true;
        return num(nullptr);
    }
};

struct Head {
    std::string format, params_file, sha, activation = "gelu";
    double version = -1, nparam = -1, nfeat = -1, hidden = -1, k0 = -1;
    std::vector<double> lo, hi;
};

bool parse_head(const std::string& text, Head& h) {
    Json j{text.data(), text.data() + text.size()};
    j.ws();
    if (j.p >= j.e || *j.p != '{') return false;
    ++j.p;
    j.ws();
    if (j.p < j.e && *j.p == '}') return false;
    for (;;) {
        std::string key;
        if (!j.str(&key)) return false;
        j.ws();
        if (j.p >= j.e || *j.p != ':') return false;
        ++j.p;
        j.ws();
        if (key == "format" || key == "params_file" || key == "params_sha256" || key == "activation") {
            std::string v;
            if (!j.str(&v)) return false;
            (key == "format" ? h.format : key == "params_file" ? h.params_file
                                         : key == "activation" ? h.activation : h.sha) = v;
        } else if (key == "version" || key == "nparam" || key == "nfeat" || key == "hidden" || key == "k0") {
            double v;
            if (!j.num(&v)) return false;
            (key == "version" ? h.version : key == "nparam" ? h.nparam : key == "nfeat" ? h.nfeat
                                                              : key == "hidden" ? h.hidden : h.k0) = v;
        } else if (key == "feature_lo" || key == "feature_hi") {
            std::vector<double>& a = key == "feature_lo" ? h.lo : h.hi;
            if (j.p >= j.e || *j.p != '[') return false;
            ++j.p;
            j.ws();
            if (j.p < j.e && *j.p == ']') {
                ++j.p;
            } else {
                for (;;) {
                    double v;
                    if (!j.num(&v)) return false;
                    a.push_back(v);
                    j.ws();
                    if (j.p < j.e && *j.p == ',') {
                        ++j.p;
                        continue;
                    }
                    if (j.p < j.e && *j.p == ']') {
                        ++j.p;
                        break;
                    }
                    return false;
                }
            }
        } else if (!j.skip()) {
            return false;
        }
        j.ws();
        if (j.p < j.e && *j.p == ',') {
            ++j.p;
            continue;
        }
        if (j.p < j.e && *j.p == '}') {
            ++j.p;
            break;
        }
        return false;
    }
    j.ws();
    return j.ok && j.p == j.e;
}

bool read_file(const std::string& path, std::string& out) {
    FILE* f = fopen(path.c_str(), "rb");
    if (!f) return false;
    char buf[1 << 16];
    size_t k;
    out.clear();
    while ((k = fread(buf, 1, sizeof buf, f)) > 0) out.append(buf, k);
    const bool ok = !ferror(f);
    fclose(f);
    return ok;
}

bool write_file(const std::string& path, const void* data, size_t len) {
    FILE* f = fopen(path.c_str(), "wb");
    if (!f) return false;
    const bool ok = fwrite(data, 1, len, f) == len;
    return fclose(f) == 0 && ok;
}

std::string base_name(const std::string& path) {
    const size_t k = path.find_last_of('/');
    return k == std::string::npos ? path : path.substr(k + 1);
}

std::string dir_name(const std::string& path) {
    const size_t k = path.find_last_of('/');
    return k == std::string::npos ? std::string() : path.substr(0, k + 1);
}

constexpr const char* kFormat = "dual-grid drag closure";
constexpr int kVersion = 1;
constexpr int kHidden = 64;   // the network's hidden width and padded input width (include/cg.h)
constexpr int kK0 = 16;

bool finite_box(const float* lo, const float* hi) {
    for (int k = 0; k < CG_MLP_NFEAT; ++k)
        if (!std::isfinite(lo[k]) || !std::isfinite(hi[k]) || !(hi[k] > lo[k])) return false;
    return true;
}

}  // namespace

extern "C" {

cg_status cg_mlp_checkpoint_write(const char* path, const float* params, const float* feat_lo, const float* feat_hi,
                                  int32_t activation, const char* meta_json) {
    if (!path || !*path || !params || !feat_lo || !feat_hi) return CG_ERR_INVALID_ARG;
    if (activation != CG_MLP_GELU && activation != CG_MLP_RELU) return CG_ERR_INVALID_ARG;
    for (int k = 0; k < CG_MLP_NPARAM; ++k)
        if (!std::isfinite(params[k])) return CG_ERR_INVALID_ARG;
    if (!finite_box(feat_lo, feat_hi)) return CG_ERR_INVALID_ARG;
    std::string meta = meta_json ? meta_json : "{}";
    {
        Json j{meta.data(), meta.data() + meta.size()};
        j.ws();
        if (j.p >= j.e || *j.p != '{' || !j.skip()) return CG_ERR_INVALID_ARG;
        j.ws();
        if (j.p != j.e) return CG_ERR_INVALID_ARG;
    }
    // little-endian float32 bytes, whatever the host's order
    std::vector<unsigned char> raw(4 * (size_t)CG_MLP_NPARAM);
    for (int k = 0; k < CG_MLP_NPARAM; ++k) {
        uint32_t u;
        memcpy(&u, &params[k], 4);
        for (int b = 0; b < 4; ++b) raw[4 * (size_t)k + b] = (unsigned char)(u >> (8 * b));
    }
    const std::string p(path);
    std::string head = "{\n \"format\": \"" + std::string(kFormat) + "\",\n \"version\": " + std::to_string(kVersion) +
                       ",\n \"nparam\": " + std::to_string(CG_MLP_NPARAM) + ",\n \"nfeat\": " +
                       std::to_string(CG_MLP_NFEAT) + ",\n \"hidden\": " + std::to_string(kHidden) + ",\n \"k0\": " +
                       std::to_string(kK0) + ",\n \"params_file\": \"" + base_name(p) + ".f32\",\n \"params_sha256\": \"" +
                       sha256_hex(raw.data(), raw.size()) + "\",\n";
    auto arr = [&](const char* name, const float* v) {
        std::string s = std::string(" \"") + name + "\": [";
        char buf[40];
        for (int k = 0; k < CG_MLP_NFEAT; ++k) {
            snprintf(buf, sizeof buf, "%.17g", (double)v[k]);   // the float's exact value, round-tripped
            s += (k ? ", " : "") + std::string(buf);
        }
        return s + "],\n";
    };
    head += arr("feature_lo", feat_lo) + arr("feature_hi", feat_hi) + " \"activation\": \"" +
            (activation == CG_MLP_RELU ? "relu" : "gelu") + "\",\n \"meta\": " + meta + "\n}\n";
    if (!write_file(p + ".f32", raw.data(), raw.size())) return CG_ERR_INVALID_ARG;
    if (!write_file(p + ".json", head.data(), head.size())) return CG_ERR_INVALID_ARG;
    return CG_OK;
}

cg_status cg_mlp_checkpoint_read(const char* path, float* params, float* feat_lo, float* feat_hi,
                                 int32_t* activation) {
    if (!path || !*path) return CG_ERR_INVALID_ARG;
    const std::string p(path);
    std::string text, raw;
    Head h;
    if (!read_file(p + ".json", text) || !parse_head(text, h)) return CG_ERR_INVALID_ARG;
    if (h.format != kFormat || h.version != kVersion) return CG_ERR_INVALID_ARG;
    if (h.nparam != CG_MLP_NPARAM || h.nfeat != CG_MLP_NFEAT || h.hidden != kHidden || h.k0 != kK0)
        return CG_ERR_INVALID_ARG;
    if (h.params_file.empty() || h.params_file.find('/') != std::string::npos) return CG_ERR_INVALID_ARG;
    if ((int)h.lo.size() != CG_MLP_NFEAT || (int)h.hi.size() != CG_MLP_NFEAT) return CG_ERR_INVALID_ARG;
    if (h.activation != "gelu" && h.activation != "relu") return CG_ERR_INVALID_ARG;
    if (!read_file(dir_name(p) + h.params_file, raw) || raw.size() != 4 * (size_t)CG_MLP_NPARAM) return CG_ERR_INVALID_ARG;
    if (sha256_hex((const unsigned char*)raw.data(), raw.size()) != h.sha) return CG_ERR_INVALID_ARG;
    float P[CG_MLP_NPARAM], lo[CG_MLP_NFEAT], hi[CG_MLP_NFEAT];
    for (int k = 0; k < CG_MLP_NPARAM; ++k) {
        uint32_t u = 0;
        for (int b = 0; b < 4; ++b) u |= (uint32_t)(unsigned char)raw[4 * (size_t)k + b] << (8 * b);
        memcpy(&P[k], &u, 4);
        if (!std::isfinite(P[k])) return CG_ERR_INVALID_ARG;
    }
    for (int k = 0; k < CG_MLP_NFEAT; ++k) {
        lo[k] = (float)h.lo[k];
        hi[k] = (float)h.hi[k];
    }
    if (!finite_box(lo, hi)) return CG_ERR_INVALID_ARG;
    if (params) memcpy(params, P, sizeof P);
    if (feat_lo) memcpy(feat_lo, lo, sizeof lo);
    if (feat_hi) memcpy(feat_hi, hi, sizeof hi);
    if (activation) *activation = h.activation == "relu" ? CG_MLP_RELU : CG_MLP_GELU;
    return CG_OK;
}

cg_status cg_mlp_save(cg_mlp* m, const char* path, const char* meta_json) {
    if (!m || !path) return CG_ERR_INVALID_ARG;
    float P[CG_MLP_NPARAM], lo[CG_MLP_NFEAT], hi[CG_MLP_NFEAT];
    CG_TRY(cg_mlp_get_params(m, P, nullptr));
    int32_t act = CG_MLP_GELU;
    CG_TRY(cg::mlp_feature_box(m, lo, hi));
    CG_TRY(cg_mlp_get_activation(m, &act));
    return cg_mlp_checkpoint_write(path, P, lo, hi, act, meta_json);
}

cg_status cg_mlp_load(const char* path, void* cuda_stream, cg_mlp** out) {
    if (!out) return CG_ERR_INVALID_ARG;
    *out = nullptr;
    float P[CG_MLP_NPARAM], lo[CG_MLP_NFEAT], hi[CG_MLP_NFEAT];
    int32_t act = CG_MLP_GELU;
    CG_TRY(cg_mlp_checkpoint_read(path, P, lo, hi, &act));
    CG_TRY(cg_mlp_create(P, lo, hi, cuda_stream, out));
    const cg_status s = cg_mlp_set_activation(*out, act);
    if (s != CG_OK) {
        cg_mlp_destroy(*out);
        *out = nullptr;
    }
    return s;
}

}  // extern "C"
