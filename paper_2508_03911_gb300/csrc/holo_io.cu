// holo_io.cu -- reader and writer of .holo files (the paper's "Holofile system"
// section): 64-byte header, frames as one binary stream, optional JSON footer.
// Host code; device destinations are filled through a pinned bounce buffer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hv.h"

namespace {

constexpr size_t kHeader = 64;
constexpr uint16_t kVersion = 7;

// Little-endian field access (independent of the host's byte order).
uint64_t get_le(const unsigned char* p, int n) {
  uint64_t v = 0;
  for (int i = n - 1; i >= 0; --i) v = (v << 8) | p[i];
  return v;
}
void put_le(unsigned char* p, uint64_t v, int n) {
  for (int i = 0; i < n; ++i) p[i] = static_cast<unsigned char>(v >> (8 * i));
}

struct File {
  FILE* f = nullptr;
  explicit File(const char* path, const char* mode) : f(path ? std::fopen(path, mode) : nullptr) {}
  ~File() {
    if (f) std::fclose(f);
  }
};

bool file_size(FILE* f, uint64_t* size) {
  if (std::fseek(f, 0, SEEK_END) != 0) return false;
  const long s = std::ftell(f);
  if (s < 0) return false;
  *size = uint64_t(s);
  return std::fseek(f, 0, SEEK_SET) == 0;
}

hv_status parse(FILE* f, hv_holo_header* h, uint64_t* fsize) {
  if (!file_size(f, fsize) || *fsize < kHeader) return HV_ERR_ARG;
  unsigned char b[kHeader];
  if (std::fread(b, 1, kHeader, f) != kHeader) return HV_ERR_ARG;
  if (std::memcmp(b, "HOLO", 4) != 0) return HV_ERR_ARG;
  hv_holo_header r{};
  r.version = uint16_t(get_le(b + 4, 2));
  r.bits_per_pixel = uint16_t(get_le(b + 6, 2));
  r.width = uint32_t(get_le(b + 8, 4));
  r.height = uint32_t(get_le(b + 12, 4));
  r.n_images = uint32_t(get_le(b + 16, 4));
  r.data_bytes = get_le(b + 20, 8);
  r.endianness = b[28];
  r.data_type = b[29];
  if (r.version != kVersion) return HV_ERR_UNSUPPORTED;
  if (r.bits_per_pixel == 0 || r.bits_per_pixel % 8 != 0 || r.endianness > 1 || r.data_type > 1) return HV_ERR_ARG;
  const uint64_t want = uint64_t(r.n_images) * r.width * r.height * (r.bits_per_pixel / 8);
  if (r.data_bytes != want || kHeader + r.data_bytes > *fsize) return HV_ERR_ARG;
  *h = r;
  return HV_OK;
}

void swap_bytes(unsigned char* p, size_t count, int bpp) {
  for (size_t i = 0; i < count; ++i, p += bpp)
    for (int a = 0, b = bpp - 1; a < b; ++a, --b) std::swap(p[a], p[b]);
}

}  // namespace

extern "C" {

hv_status hv_holo_read_header(const char* path, hv_holo_header* hdr) {
  if (!path || !hdr) return HV_ERR_ARG;
  File f(path, "rb");
  if (!f.f) return HV_ERR_ARG;
  uint64_t fsize = 0;
  return parse(f.f, hdr, &fsize);
}

hv_status hv_holo_read_frames(const char* path, uint64_t first, uint32_t n, void* dst, int mem_kind, void* stream) {
  if (!path || !dst || (mem_kind != HV_MEM_HOST && mem_kind != HV_MEM_DEVICE)) return HV_ERR_ARG;
  File f(path, "rb");
  if (!f.f) return HV_ERR_ARG;
  hv_holo_header h{};
  uint64_t fsize = 0;
  hv_status s = parse(f.f, &h, &fsize);
  if (s != HV_OK) return s;
  if (n == 0) return HV_OK;
  if (first + n > h.n_images) return HV_ERR_ARG;
  const int bpp = h.bits_per_pixel / 8;
  const uint64_t fb = uint64_t(h.width) * h.height * bpp;
  if (std::fseek(f.f, long(kHeader + first * fb), SEEK_SET) != 0) return HV_ERR_ARG;
  const bool swap = h.endianness == 1 && bpp > 1;
  if (mem_kind == HV_MEM_HOST) {
    unsigned char* d = static_cast<unsigned char*>(dst);
    if (std::fread(d, 1, size_t(fb * n), f.f) != size_t(fb * n)) return HV_ERR_ARG;
    if (swap) swap_bytes(d, size_t(uint64_t(h.width) * h.height * n), bpp);
    return HV_OK;
  }
  // device: two pinned halves of about 32 MiB, read one while the other copies
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t per = std::max<uint64_t>(1, (uint64_t(32) << 20) / fb);
  unsigned char* pin = nullptr;
  if (cudaMallocHost(&pin, size_t(2 * per * fb)) != cudaSuccess) return HV_ERR_CUDA;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e = cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
  s = e == cudaSuccess ? HV_OK : HV_ERR_CUDA;
  unsigned char* d = static_cast<unsigned char*>(dst);
  int k = 0;
  for (uint64_t a = 0; a < n && s == HV_OK; a += per, k ^= 1) {
    const uint64_t m = std::min<uint64_t>(per, n - a);
    unsigned char* half = pin + k * per * fb;
    if (cudaEventSynchronize(ev[k]) != cudaSuccess) {  // its previous copy is done
      s = HV_ERR_CUDA;
      break;
    }
    if (std::fread(half, 1, size_t(m * fb), f.f) != size_t(m * fb)) {
      s = HV_ERR_ARG;
      break;
    }
    if (swap) swap_bytes(half, size_t(uint64_t(h.width) * h.height * m), bpp);
    if (cudaMemcpyAsync(d + a * fb, half, size_t(m * fb), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaEventRecord(ev[k], st) != cudaSuccess)
      s = HV_ERR_CUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && s == HV_OK) s = HV_ERR_CUDA;
  for (auto x : ev)
    if (x) cudaEventDestroy(x);
  cudaFreeHost(pin);
  return s;
}

hv_status hv_holo_read_footer(const char* path, char* buf, size_t cap, size_t* len) {
  if (!path || !len) return HV_ERR_ARG;
  File f(path, "rb");
  if (!f.f) return HV_ERR_ARG;
  hv_holo_header h{};
  uint64_t fsize = 0;
  hv_status s = parse(f.f, &h, &fsize);
  if (s != HV_OK) return s;
  const uint64_t off = kHeader + h.data_bytes;
  *len = size_t(fsize - off);
  if (!buf) return HV_OK;
  if (cap <= *len) return HV_ERR_ARG;
  if (std::fseek(f.f, long(off), SEEK_SET) != 0) return HV_ERR_ARG;
  if (std::fread(buf, 1, *len, f.f) != *len) return HV_ERR_ARG;
  buf[*len] = '\0';
  return HV_OK;
}

hv_status hv_holo_write(const char* path, const hv_holo_header* hdr, const void* frames, const char* footer_json) {
  if (!path || !hdr || (!frames && hdr->n_images > 0)) return HV_ERR_ARG;
  if (hdr->bits_per_pixel == 0 || hdr->bits_per_pixel % 8 != 0 || hdr->endianness != 0 || hdr->data_type > 1)
    return HV_ERR_ARG;
  const uint64_t bytes = uint64_t(hdr->n_images) * hdr->width * hdr->height * (hdr->bits_per_pixel / 8);
  unsigned char b[kHeader] = {};
  std::memcpy(b, "HOLO", 4);
  put_le(b + 4, kVersion, 2);
  put_le(b + 6, hdr->bits_per_pixel, 2);
  put_le(b + 8, hdr->width, 4);
  put_le(b + 12, hdr->height, 4);
  put_le(b + 16, hdr->n_images, 4);
  put_le(b + 20, bytes, 8);
  b[28] = 0;
  b[29] = hdr->data_type;
  File f(path, "wb");
  if (!f.f) return HV_ERR_ARG;
  if (std::fwrite(b, 1, kHeader, f.f) != kHeader) return HV_ERR_ARG;
  if (bytes && std::fwrite(frames, 1, size_t(bytes), f.f) != size_t(bytes)) return HV_ERR_ARG;
  if (footer_json) {
    const size_t L = std::strlen(footer_json);
    if (std::fwrite(footer_json, 1, L, f.f) != L) return HV_ERR_ARG;
  }
  return HV_OK;
}

}  // extern "C"
