// MPI_Info-style hint objects and MPIX_Info_set_hex (§3.2: passing opaque
// binary info hints).  An info object is an ordered set of (key, value)
// strings.  A binary value (a cudaStream_t, say) is stored as text: two
// lowercase hexadecimal digits per byte, bytes in memory order.  The paper
// leaves the encoding to the implementation and proposes the setter only;
// mpx_info_get_hex is the matching reader it calls for "for completeness".
// Host-only code: nothing here touches the GPU.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "mpx.h"

struct mpx_info_s {
  std::mutex mu;
  std::vector<std::pair<std::string, std::string>> kv;  // in insertion order
};

namespace {

bool key_ok(const char* key) {
  if (!key) return false;
  const size_t n = strnlen(key, MPX_MAX_INFO_KEY + 1);
  return n >= 1 && n <= MPX_MAX_INFO_KEY;
}

std::string* find(mpx_info_s* info, const char* key) {
  for (auto& e : info->kv)
    if (e.first == key) return &e.second;
  return nullptr;
}

int hex_digit(char c) {
  if (c >= '0' && c <= '9') return c - '0';
  if (c >= 'a' && c <= 'f') return c - 'a' + 10;
  if (c >= 'A' && c <= 'F') return c - 'A' + 10;
  return -1;
}

}  // namespace

extern "C" int mpx_info_create(mpx_info_t* info) {
  if (!info) return MPX_ERR_ARG;
  *info = new (std::nothrow) mpx_info_s();
  return *info ? MPX_SUCCESS : MPX_ERR_NO_MEM;
}

extern "C" int mpx_info_free(mpx_info_t* info) {
  if (!info || !*info) return MPX_ERR_ARG;
  delete *info;
  *info = nullptr;
  return MPX_SUCCESS;
}

extern "C" int mpx_info_set(mpx_info_t info, const char* key, const char* value) {
  if (!info || !key_ok(key) || !value) return MPX_ERR_ARG;
  if (strnlen(value, MPX_MAX_INFO_VAL + 1) > MPX_MAX_INFO_VAL) return MPX_ERR_ARG;
  std::lock_guard<std::mutex> g(info->mu);
  if (std::string* v = find(info, key)) {
    *v = value;
  } else {
    info->kv.emplace_back(key, value);
  }
  return MPX_SUCCESS;
}

extern "C" int mpx_info_get(mpx_info_t info, const char* key, char* value, int buflen, int* flag) {
  if (!info || !key_ok(key) || !flag || (buflen > 0 && !value) || buflen < 0) return MPX_ERR_ARG;
  std::lock_guard<std::mutex> g(info->mu);
  const std::string* v = find(info, key);
  *flag = v != nullptr;
  if (v && buflen > 0) {
    const size_t n = std::min(v->size(), (size_t)buflen - 1);
    memcpy(value, v->data(), n);
    value[n] = '\0';
  }
  return MPX_SUCCESS;
}

extern "C" int mpx_info_get_valuelen(mpx_info_t info, const char* key, int* valuelen, int* flag) {
  if (!info || !key_ok(key) || !valuelen || !flag) return MPX_ERR_ARG;
  std::lock_guard<std::mutex> g(info->mu);
  const std::string* v = find(info, key);
  *flag = v != nullptr;
  *valuelen = v ? (int)v->size() : 0;
  return MPX_SUCCESS;
}

extern "C" int mpx_info_get_nkeys(mpx_info_t info, int* nkeys) {
  if (!info || !nkeys) return MPX_ERR_ARG;
  std::lock_guard<std::mutex> g(info->mu);
  *nkeys = (int)info->kv.size();
  return MPX_SUCCESS;
}

extern "C" int mpx_info_get_nthkey(mpx_info_t info, int n, char* key, int buflen) {
  if (!info || !key || buflen < 1) return MPX_ERR_ARG;
  std::lock_guard<std::mutex> g(info->mu);
  if (n < 0 || n >= (int)info->kv.size()) return MPX_ERR_ARG;
  const std::string& k = info->kv[(size_t)n].first;
  const size_t len = std::min(k.size(), (size_t)buflen - 1);
  memcpy(key, k.data(), len);
  key[len] = '\0';
  return MPX_SUCCESS;
}

extern "C" int mpx_info_set_hex(mpx_info_t info, const char* key, const void* value, int vallen) {
  if (!info || !key_ok(key) || !value || vallen < 1 || 2 * (int64_t)vallen > MPX_MAX_INFO_VAL)
    return MPX_ERR_ARG;
  static const char digits[] = "0123456789abcdef";
  const uint8_t* b = static_cast<const uint8_t*>(value);
  std::string text((size_t)vallen * 2, '0');
  for (int i = 0; i < vallen; ++i) {
    text[2 * (size_t)i] = digits[b[i] >> 4];
    text[2 * (size_t)i + 1] = digits[b[i] & 15];
  }
  return mpx_info_set(info, key, text.c_str());
}

extern "C" int mpx_info_get_hex(mpx_info_t info, const char* key, void* value, int vallen, int* flag) {
  if (!info || !key_ok(key) || !value || vallen < 1 || !flag) return MPX_ERR_ARG;
  std::lock_guard<std::mutex> g(info->mu);
  const std::string* v = find(info, key);
  *flag = v != nullptr;
  if (!v) return MPX_SUCCESS;
  if (v->size() != 2 * (size_t)vallen) return MPX_ERR_ARG;  // not a value of this length
  uint8_t* out = static_cast<uint8_t*>(value);
  std::vector<uint8_t> tmp((size_t)vallen);
  for (int i = 0; i < vallen; ++i) {
    const int hi = hex_digit((*v)[2 * (size_t)i]), lo = hex_digit((*v)[2 * (size_t)i + 1]);
    if (hi < 0 || lo < 0) return MPX_ERR_ARG;
    tmp[(size_t)i] = (uint8_t)(hi << 4 | lo);
  }
  memcpy(out, tmp.data(), (size_t)vallen);
  return MPX_SUCCESS;
}
