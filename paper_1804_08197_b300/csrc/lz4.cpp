// LZ4 block format ("Volumetric Data Storage": chunks are LZ4-compressed),
// written from the format's published definition. A block is a series of
// sequences; each sequence is a token byte (high nibble: literal count, low
// nibble: match length - 4; 15 means more length bytes follow, each adding
// up to 255, the first byte below 255 ending the run), the literals, then a
// 2-byte little-endian match offset (1..65535) and the optional match length
// bytes. The last sequence has literals only. Rules the encoder keeps (the
// decoder checks bounds instead of relying on them): the last 5 bytes are
// literals and the last match starts at least 12 bytes before the end.
#include <stdint.h>
#include <string.h>

#include <vector>

#include "internal.h"

namespace sg {

size_t lz4_bound(size_t n) { return n + n / 255 + 16; }

namespace {

constexpr int kMinMatch = 4;
constexpr int kLastLiterals = 5;
constexpr int kMatchGuard = 12;
constexpr int kHashBits = 16;

inline uint32_t read32(const uint8_t* p) {
  uint32_t v;
  memcpy(&v, p, 4);
  return v;
}

inline uint32_t hash4(uint32_t v) { return (v * 2654435761u) >> (32 - kHashBits); }

// writes a length continuation (the part beyond the nibble's 15)
inline uint8_t* put_length(uint8_t* op, size_t len) {
  while (len >= 255) {
    *op++ = 255;
    len -= 255;
  }
  *op++ = (uint8_t)len;
  return op;
}

}  // namespace

// Greedy single-pass encoder with a 2^16-entry hash of 4-byte sequences.
// Returns the compressed size (<= lz4_bound(n)).
size_t lz4_compress(const uint8_t* src, size_t n, uint8_t* dst) {
  uint8_t* op = dst;
  const uint8_t* anchor = src;  // first literal not yet emitted
  if (n >= (size_t)kMatchGuard + 1) {
    std::vector<uint32_t> table((size_t)1 << kHashBits, 0xffffffffu);
    const uint8_t* const match_limit = src + n - kMatchGuard;   // a match must start before this
    const uint8_t* const end_limit = src + n - kLastLiterals;   // and end at or before this
    const uint8_t* ip = src;
    while (ip < match_limit) {
      const uint32_t seq = read32(ip);
      const uint32_t h = hash4(seq);
      const uint32_t cand = table[h];
      table[h] = (uint32_t)(ip - src);
      if (cand == 0xffffffffu || (size_t)(ip - src) - cand > 65535 || read32(src + cand) != seq) {
        ++ip;
        continue;
      }
      const uint8_t* ref = src + cand;
      // extend the match forwards (not past end_limit)
      const uint8_t* mp = ip + kMinMatch;
      const uint8_t* rp = ref + kMinMatch;
      while (mp < end_limit && *mp == *rp) {
        ++mp;
        ++rp;
      }
      const size_t lit = (size_t)(ip - anchor), mlen = (size_t)(mp - ip) - kMinMatch;
      uint8_t* token = op++;
      *token = (uint8_t)((lit >= 15 ? 15 : lit) << 4);
      if (lit >= 15) op = put_length(op, lit - 15);
      memcpy(op, anchor, lit);
      op += lit;
      const uint32_t off = (uint32_t)(ip - ref);
      *op++ = (uint8_t)(off & 255);
      *op++ = (uint8_t)(off >> 8);
      *token |= (uint8_t)(mlen >= 15 ? 15 : mlen);
      if (mlen >= 15) op = put_length(op, mlen - 15);
      ip = mp;
      anchor = ip;
    }
  }
  // last literals
  const size_t lit = (size_t)(src + n - anchor);
  uint8_t* token = op++;
  *token = (uint8_t)((lit >= 15 ? 15 : lit) << 4);
  if (lit >= 15) op = put_length(op, lit - 15);
  memcpy(op, anchor, lit);
  op += lit;
  return (size_t)(op - dst);
}

// Decodes a block of csize bytes into exactly n bytes. Returns false on any
// malformed input (out-of-range offset, overrun of either buffer, wrong
// output size); never reads or writes outside the two buffers.
bool lz4_decompress(const uint8_t* src, size_t csize, uint8_t* dst, size_t n) {
  const uint8_t* ip = src;
  const uint8_t* const iend = src + csize;
  uint8_t* op = dst;
  uint8_t* const oend = dst + n;
  while (ip < iend) {
    const uint8_t token = *ip++;
    size_t lit = token >> 4;
    if (lit == 15) {
      uint8_t b;
      do {
        if (ip >= iend) return false;
        b = *ip++;
        lit += b;
      } while (b == 255);
    }
    if (lit > (size_t)(iend - ip) || lit > (size_t)(oend - op)) return false;
    memcpy(op, ip, lit);
    ip += lit;
    op += lit;
    if (ip == iend) break;  // the last sequence carries literals only
    if (iend - ip < 2) return false;
    const size_t off = (size_t)ip[0] | ((size_t)ip[1] << 8);
    ip += 2;
    if (off == 0 || off > (size_t)(op - dst)) return false;
    size_t mlen = token & 15;
    if (mlen == 15) {
      uint8_t b;
      do {
        if (ip >= iend) return false;
        b = *ip++;
        mlen += b;
      } while (b == 255);
    }
    mlen += kMinMatch;
    if (mlen > (size_t)(oend - op)) return false;
    const uint8_t* ref = op - off;
    for (size_t i = 0; i < mlen; ++i) op[i] = ref[i];  // overlapping copies repeat the pattern
    op += mlen;
  }
  return op == oend;
}

}  // namespace sg
