// Network checkpoints in the C ABI (unet_save / unet_load, include/unet.h): a trained
// U-Net's FP32 master weights and BatchNorm running statistics -- the state the
// preconditioners of Sec. 3 read -- written to a file and restored, so that a network
// trained once serves many solves.  Host code only.
//
// File layout (little-endian):
//   8 bytes   magic "HLMUNET1"
//   4 bytes   uint32 length L of the JSON header
//   L bytes   JSON object: "cfg" (the unet_cfg fields), "crc32" (of the payload),
//             "meta" (the caller's JSON object), "n_bn", "n_params", "version" (1)
//   padding   zeros up to a multiple of 16 bytes
//   payload   float32[n_params] weights in the flat order of include/unet.h, then
//             float32[n_bn] BatchNorm running means and variances
// The reader parses the header as JSON (any key order and spacing), so files written
// by other tools in this layout load too.  Adam moments are not stored.
#include <array>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/helm.h"
#include "../../include/unet.h"
#include "unet_api.h"

namespace helm {
void set_error(const std::string& s);
}

namespace {

constexpr char kMagic[8] = {'H', 'L', 'M', 'U', 'N', 'E', 'T', '1'};
constexpr int kVersion = 1;

// CRC-32 of the IEEE 802.3 polynomial in its reflected form 0xEDB88320, initial value
// and final XOR 0xFFFFFFFF (the checksum zlib's crc32 computes), table driven.
uint32_t crc32_of(const unsigned char* p, size_t n) {
  static const std::array<uint32_t, 256> table = [] {
    std::array<uint32_t, 256> t{};
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int k = 0; k < 8; ++k) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
      t[i] = c;
    }
    return t;
  }();
  uint32_t c = 0xFFFFFFFFu;
  for (size_t i = 0; i < n; ++i) c = table[(c ^ p[i]) & 0xFFu] ^ (c >> 8);
  return c ^ 0xFFFFFFFFu;
}

// A small JSON reader: objects, arrays, strings, numbers, true / false / null.
struct JVal {
  enum Kind { Null, Bool, Num, Str, Arr, Obj } kind = Null;
  double num = 0;
  std::string str;
  std::vector<JVal> arr;
  std::map<std::string, JVal> obj;
  std::string raw;   // the value's source text (to carry "meta" through unchanged)
};

struct JParser {
  const char* s;
  size_t n, i = 0;
  bool ok = true;
  JParser(const char* text, size_t len) : s(text), n(len) {}
  void ws() {
    while (i < n && (s[i] == ' ' || s[i] == '\t' || s[i] == '\n' || s[i] == '\r')) ++i;
  }
  bool lit(const char* w) {
    size_t k = strlen(w);
    if (i + k <= n && strncmp(s + i, w, k) == 0) { i += k; return true; }
    return false;
  }
  std::string string() {
    std::string out;
    if (i >= n || s[i] != '"') { ok = false; return out; }
    ++i;
    while (i < n && s[i] != '"') {
      if (s[i] == '\\') {
        if (i + 1 >= n) { ok = false; return out; }
        const char e = s[i + 1];
        if (e == 'u') {            // kept as written: keys and values read here are ASCII
          if (i + 6 > n) { ok = false; return out; }
          out.append(s + i, 6);
          i += 6;
          continue;
        }
        const char* from = "\"\\/bfnrt";
        const char* to = "\"\\/\b\f\n\r\t";
        const char* q = strchr(from, e);
        if (!q || !*q) { ok = false; return out; }
        out.push_back(to[q - from]);
        i += 2;
      } else {
        out.push_back(s[i++]);
      }
    }
    if (i >= n) { ok = false; return out; }
    ++i;
    return out;
  }
  JVal value(int depth = 0) {
    JVal v;
    if (depth > 64) { ok = false; return v; }
    ws();
    const size_t start = i;
    if (i >= n) { ok = false; return v; }
    if (s[i] == '{') {
      v.kind = JVal::Obj;
      ++i;
      ws();
      if (i < n && s[i] == '}') { ++i; }
      else {
        for (;;) {
          ws();
          std::string k = string();
          if (!ok) return v;
          ws();
          if (i >= n || s[i] != ':') { ok = false; return v; }
          ++i;
          v.obj[k] = value(depth + 1);
          if (!ok) return v;
          ws();
          if (i < n && s[i] == ',') { ++i; continue; }
          if (i < n && s[i] == '}') { ++i; break; }
          ok = false;
          return v;
        }
      }
    } else if (s[i] == '[') {
      v.kind = JVal::Arr;
      ++i;
      ws();
      if (i < n && s[i] == ']') { ++i; }
      else {
        for (;;) {
          v.arr.push_back(value(depth + 1));
          if (!ok) return v;
          ws();
          if (i < n && s[i] == ',') { ++i; continue; }
          if (i < n && s[i] == ']') { ++i; break; }
          ok = false;
          return v;
        }
      }
    } else if (s[i] == '"') {
      v.kind = JVal::Str;
      v.str = string();
    } else if (lit("true")) {
      v.kind = JVal::Bool; v.num = 1;
    } else if (lit("false")) {
      v.kind = JVal::Bool; v.num = 0;
    } else if (lit("null")) {
      v.kind = JVal::Null;
    } else {
      char* end = nullptr;
      std::string tok;
      while (i < n && strchr("+-0123456789.eE", s[i])) tok.push_back(s[i++]);
      if (tok.empty()) { ok = false; return v; }
      v.kind = JVal::Num;
      v.num = strtod(tok.c_str(), &end);
      if (!end || *end) { ok = false; return v; }
    }
    v.raw.assign(s + start, i - start);
    return v;
  }
};

bool as_int(const JVal& v, long long& out) {
  if (v.kind != JVal::Num || v.num != (double)(long long)v.num) return false;
  out = (long long)v.num;
  return true;
}

// The unet_cfg fields as a JSON object (keys sorted, like the Python writer).
std::string cfg_json(const unet_cfg& c) {
  auto arr = [](const int* a, int n) {
    std::string s = "[";
    for (int i = 0; i < n; ++i) s += (i ? ", " : "") + std::to_string(a[i]);
    return s + "]";
  };
  return "{\"coarse_resnets\": " + std::to_string(c.coarse_resnets) + ", \"context\": " + arr(c.context, 9) +
         ", \"flags\": " + std::to_string(c.flags) + ", \"in_ch\": " + std::to_string(c.in_ch) +
         ", \"levels\": " + std::to_string(c.levels) + ", \"out_ch\": " + std::to_string(c.out_ch) +
         ", \"widths\": " + arr(c.widths, 8) + "}";
}

bool cfg_matches(const JVal& j, const unet_cfg& c, std::string& why) {
  if (j.kind != JVal::Obj) { why = "cfg is not an object"; return false; }
  auto scalar = [&](const char* k, int want) {
    auto it = j.obj.find(k);
    long long v;
    if (it == j.obj.end() || !as_int(it->second, v)) { why = std::string("cfg field ") + k + " missing"; return false; }
    if (v != want) {
      why = std::string("cfg field ") + k + " is " + std::to_string(v) + ", the network's is " + std::to_string(want);
      return false;
    }
    return true;
  };
  auto array = [&](const char* k, const int* want, int n) {
    auto it = j.obj.find(k);
    if (it == j.obj.end() || it->second.kind != JVal::Arr || (int)it->second.arr.size() != n) {
      why = std::string("cfg field ") + k + " missing or of the wrong length";
      return false;
    }
    for (int i = 0; i < n; ++i) {
      long long v;
      if (!as_int(it->second.arr[i], v) || v != want[i]) {
        why = std::string("cfg field ") + k + " differs from the network's";
        return false;
      }
    }
    return true;
  };
  return scalar("in_ch", c.in_ch) && scalar("out_ch", c.out_ch) && scalar("levels", c.levels) &&
         scalar("coarse_resnets", c.coarse_resnets) && scalar("flags", c.flags) && array("widths", c.widths, 8) &&
         array("context", c.context, 9);
}

struct FileCloser {
  void operator()(FILE* f) const { if (f) fclose(f); }
};

}  // namespace

extern "C" {

int unet_save(unet_t net, const char* path, const char* meta_json) {
  if (!net || !path) { helm::set_error("unet_save: bad arguments"); return HELM_EINVAL; }
  std::string meta = meta_json ? meta_json : "{}";
  {
    JParser p(meta.data(), meta.size());
    JVal m = p.value();
    p.ws();
    if (!p.ok || p.i != meta.size() || m.kind != JVal::Obj) {
      helm::set_error("unet_save: meta is not one JSON object");
      return HELM_EINVAL;
    }
  }
  long long np = 0, nb = 0;
  int r = unet_sizes(net, &np, &nb);
  if (r < 0) return r;
  std::vector<float> payload((size_t)(np + nb));
  if ((r = unet_get_params(net, payload.data(), np)) < 0) return r;
  if ((r = unet_get_bn_stats(net, payload.data() + np, nb)) < 0) return r;
  const unsigned char* bytes = reinterpret_cast<const unsigned char*>(payload.data());
  const size_t nbytes = payload.size() * sizeof(float);
  unet_cfg cfg{};
  unet_cfg_of(net, &cfg);
  const std::string header = "{\"cfg\": " + cfg_json(cfg) + ", \"crc32\": " + std::to_string(crc32_of(bytes, nbytes)) +
                             ", \"meta\": " + meta + ", \"n_bn\": " + std::to_string(nb) +
                             ", \"n_params\": " + std::to_string(np) + ", \"version\": " + std::to_string(kVersion) + "}";
  std::vector<unsigned char> head(kMagic, kMagic + 8);
  const uint32_t hl = (uint32_t)header.size();
  for (int k = 0; k < 4; ++k) head.push_back((unsigned char)(hl >> (8 * k)));
  head.insert(head.end(), header.begin(), header.end());
  while (head.size() % 16) head.push_back(0);
  std::unique_ptr<FILE, FileCloser> f(fopen(path, "wb"));
  if (!f) { helm::set_error(std::string("unet_save: cannot open ") + path + " for writing"); return HELM_EINVAL; }
  if (fwrite(head.data(), 1, head.size(), f.get()) != head.size() || fwrite(bytes, 1, nbytes, f.get()) != nbytes ||
      fflush(f.get()) != 0) {
    helm::set_error(std::string("unet_save: write to ") + path + " failed");
    return HELM_EINVAL;
  }
  return HELM_OK;
}

int unet_load(unet_t net, const char* path) {
  if (!net || !path) { helm::set_error("unet_load: bad arguments"); return HELM_EINVAL; }
  std::vector<unsigned char> blob;
  {
    std::unique_ptr<FILE, FileCloser> f(fopen(path, "rb"));
    if (!f) { helm::set_error(std::string("unet_load: cannot open ") + path); return HELM_EINVAL; }
    unsigned char buf[1 << 16];
    size_t k;
    while ((k = fread(buf, 1, sizeof buf, f.get())) > 0) blob.insert(blob.end(), buf, buf + k);
  }
  if (blob.size() < 12 || memcmp(blob.data(), kMagic, 8) != 0) {
    helm::set_error("unet_load: not a U-Net checkpoint (bad magic)");
    return HELM_EINVAL;
  }
  uint32_t hl = 0;
  for (int k = 0; k < 4; ++k) hl |= (uint32_t)blob[8 + k] << (8 * k);
  if ((size_t)12 + hl > blob.size()) { helm::set_error("unet_load: truncated checkpoint header"); return HELM_EINVAL; }
  JParser p(reinterpret_cast<const char*>(blob.data()) + 12, hl);
  JVal h = p.value();
  p.ws();
  if (!p.ok || p.i != hl || h.kind != JVal::Obj) { helm::set_error("unet_load: unreadable checkpoint header"); return HELM_EINVAL; }
  long long version = 0, np = 0, nb = 0, crc = 0;
  auto get = [&](const char* k, long long& v) {
    auto it = h.obj.find(k);
    return it != h.obj.end() && as_int(it->second, v);
  };
  if (!get("version", version) || version != kVersion) {
    helm::set_error("unet_load: checkpoint version " + std::to_string(version) + " (this reader: " +
                    std::to_string(kVersion) + ")");
    return HELM_EINVAL;
  }
  if (!get("n_params", np) || !get("n_bn", nb) || !get("crc32", crc) || np < 0 || nb < 0) {
    helm::set_error("unet_load: header lacks n_params, n_bn or crc32");
    return HELM_EINVAL;
  }
  size_t start = 12 + (size_t)hl;
  start += (16 - start % 16) % 16;
  if (start > blob.size() || blob.size() - start != (size_t)(np + nb) * 4) {
    helm::set_error("unet_load: payload size differs from the header's");
    return HELM_EINVAL;
  }
  if (crc32_of(blob.data() + start, blob.size() - start) != (uint32_t)crc) {
    helm::set_error("unet_load: checkpoint payload CRC mismatch");
    return HELM_EINVAL;
  }
  unet_cfg cfg{};
  unet_cfg_of(net, &cfg);
  std::string why;
  auto ci = h.obj.find("cfg");
  if (ci == h.obj.end() || !cfg_matches(ci->second, cfg, why)) {
    helm::set_error("unet_load: checkpoint configuration differs from the network's: " + why);
    return HELM_EINVAL;
  }
  long long mp = 0, mb = 0;
  int r = unet_sizes(net, &mp, &mb);
  if (r < 0) return r;
  if (mp != np || mb != nb) { helm::set_error("unet_load: checkpoint sizes differ from the network's"); return HELM_EINVAL; }
  std::vector<float> payload((size_t)(np + nb));
  memcpy(payload.data(), blob.data() + start, payload.size() * 4);
  if ((r = unet_set_params(net, payload.data(), np)) < 0) return r;
  return unet_set_bn_stats(net, payload.data() + np, nb);
}

}  // extern "C"
