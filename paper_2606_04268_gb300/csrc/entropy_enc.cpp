// Encoder of the entropy container (stream format §6), on the host: wraps an ACEAPEX stream in segments of
// at most 4096 bytes.  The stream header and block index, and each block's header and sync table, are
// stored; each block section (cmd, len, off, lit) gets its own canonical Huffman code (codes of at most 12
// bits) and is cut into segments that carry the code (the first coded one) or refer to it; a segment is
// stored when coding would not make it smaller.  A stream that does not parse is coded as one section.
//
// Code lengths: Huffman's construction (the two lightest trees merged first, ties to the tree made first,
// leaves made in symbol order), lengths above 12 cut to 12, then -- while the Kraft sum exceeds 2^12 -- the
// longest code below 12 (ties: the smaller count, then the larger symbol) lengthened by one bit.
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "../../include/aceapex.h"
#include "layout.h"

namespace {

constexpr uint32_t kSeg = 4096, kMaxLen = 12, kLanes = 32;

uint64_t le(const uint8_t *p, int n) {
    uint64_t v = 0;
    for (int i = n - 1; i >= 0; i--) v = (v << 8) | p[i];
    return v;
}
void put_le(std::vector<uint8_t> &o, uint64_t v, int n) {
    for (int i = 0; i < n; i++) o.push_back((uint8_t)(v >> (8 * i)));
}
void set_le(uint8_t *p, uint64_t v, int n) {
    for (int i = 0; i < n; i++) p[i] = (uint8_t)(v >> (8 * i));
}

struct Section {
    uint64_t begin, end;
    bool coded;
};

void code_lengths(const uint64_t *count, uint8_t *len) {
    memset(len, 0, 256);
    std::vector<uint64_t> weight(count, count + 256);
    std::vector<int> up(256, -1);
    std::vector<char> live(256);
    int used = 0;
    for (int s = 0; s < 256; s++) used += (live[s] = count[s] > 0);
    if (used == 0) return;
    if (used == 1) {
        for (int s = 0; s < 256; s++) if (count[s]) len[s] = 1;
        return;
    }
    for (int m = 0; m + 1 < used; m++) {
        int x = -1, y = -1;  // lightest, second lightest; ties keep the earlier tree
        for (int i = 0; i < (int)weight.size(); i++) {
            if (!live[i]) continue;
            if (x < 0 || weight[i] < weight[x]) { y = x; x = i; }
            else if (y < 0 || weight[i] < weight[y]) y = i;
        }
        weight.push_back(weight[x] + weight[y]);
        up.push_back(-1);
        live.push_back(1);
        up[x] = up[y] = (int)weight.size() - 1;
        live[x] = live[y] = 0;
    }
    for (int s = 0; s < 256; s++) {
        if (!count[s]) continue;
        uint32_t depth = 0;
        for (int v = s; up[v] >= 0; v = up[v]) depth++;
        len[s] = (uint8_t)(depth < kMaxLen ? depth : kMaxLen);
    }
    for (;;) {
        uint64_t kraft = 0;
        for (int s = 0; s < 256; s++) if (len[s]) kraft += 1ull << (kMaxLen - len[s]);
        if (kraft <= (1ull << kMaxLen)) return;
        int pick = -1;
        for (int s = 0; s < 256; s++) {
            if (!len[s] || len[s] >= kMaxLen) continue;
            if (pick < 0 || len[s] > len[pick] || (len[s] == len[pick] && count[s] <= count[pick])) pick = s;
        }
        len[pick]++;
    }
}

// Canonical codes: by (length, symbol), each code the previous plus one, shifted by the length difference.
void canonical(const uint8_t *len, uint32_t *code) {
    uint32_t next[kMaxLen + 2] = {0}, cnt[kMaxLen + 2] = {0};
    for (int s = 0; s < 256; s++) cnt[len[s]]++;
    cnt[0] = 0;
    uint32_t c = 0;
    for (uint32_t L = 1; L <= kMaxLen; L++) {
        c = (c + cnt[L - 1]) << 1;
        next[L] = c;
    }
    for (int s = 0; s < 256; s++) if (len[s]) code[s] = next[len[s]]++;
}

std::vector<Section> sections(const uint8_t *raw, uint64_t n) {
    std::vector<Section> out;
    auto add = [&](uint64_t a, uint64_t b, bool coded) { if (b > a) out.push_back({a, b, coded}); };
    bool ok = n >= 64 && le(raw, 4) == aceapex::kMagic;
    const uint64_t nb = ok ? le(raw + 24, 8) : 0, first = aceapex::align16(64 + 8 * nb);
    if (ok && (nb > n / 8 || first > n)) ok = false;
    std::vector<uint64_t> o_cmd(nb), o_len(nb), o_off(nb), o_lit(nb), bend(nb), boff(nb);
    for (uint64_t b = 0; ok && b < nb; b++) {
        boff[b] = le(raw + 64 + 8 * b, 8);
        bend[b] = b + 1 < nb ? le(raw + 64 + 8 * (b + 1), 8) : n;
        if ((b == 0 && boff[b] != first) || bend[b] > n || bend[b] < boff[b] + 32) { ok = false; break; }
        const uint8_t *h = raw + boff[b];
        o_cmd[b] = boff[b] + aceapex::align16(32 + 20 * le(h + 28, 4));
        o_len[b] = aceapex::align16(o_cmd[b] + le(h + 12, 4));
        o_off[b] = aceapex::align16(o_len[b] + le(h + 16, 4));
        o_lit[b] = aceapex::align16(o_off[b] + le(h + 4, 4) * h[20]);
        if (o_lit[b] > bend[b]) ok = false;
    }
    if (!ok) {
        add(0, n, true);
        return out;
    }
    add(0, first, false);
    for (uint64_t b = 0; b < nb; b++) {
        add(boff[b], o_cmd[b], false);
        add(o_cmd[b], o_len[b], true);
        add(o_len[b], o_off[b], true);
        add(o_off[b], o_lit[b], true);
        add(o_lit[b], bend[b], true);
    }
    return out;
}

}  // namespace

extern "C" int aceapex_entropy_encode(const void *raw_, size_t raw_len, void **out, size_t *out_len) {
    const uint8_t *raw = (const uint8_t *)raw_;
    if (!out || !out_len || (!raw && raw_len)) return aceapex::kErrArg;
    *out = nullptr;
    *out_len = 0;
    const std::vector<Section> secs = raw_len ? sections(raw, raw_len) : std::vector<Section>();
    uint64_t n_seg = 0;
    for (const Section &s : secs) n_seg += (s.end - s.begin + kSeg - 1) / kSeg;
    const uint64_t head = aceapex::align16(64 + 16 * n_seg);
    std::vector<uint8_t> pay;
    std::vector<uint64_t> r_off, p_off;
    for (const Section &sec : secs) {
        uint64_t count[256] = {0};
        for (uint64_t x = sec.begin; x < sec.end; x++) count[raw[x]]++;
        uint8_t len[256];
        uint32_t code[256] = {0};
        code_lengths(count, len);
        canonical(len, code);
        int64_t carrier = -1;
        for (uint64_t a = sec.begin; a < sec.end; a += kSeg) {
            const uint32_t n = (uint32_t)(sec.end - a < kSeg ? sec.end - a : kSeg);
            const uint8_t *seg = raw + a;
            r_off.push_back(a);
            p_off.push_back(head + pay.size());
            uint32_t lane_len[kLanes];
            uint64_t size = 8 + (carrier < 0 ? 128 : 0) + 2 * kLanes;
            for (uint32_t l = 0; l < kLanes; l++) {
                uint64_t bits = 0;
                for (uint32_t j = l; j < n; j += kLanes) bits += len[seg[j]];
                lane_len[l] = (uint32_t)((bits + 7) / 8);
                size += lane_len[l];
            }
            const uint64_t k = r_off.size() - 1;
            if (!sec.coded || size >= 8 + (uint64_t)n) {
                put_le(pay, 0, 8);
                pay.insert(pay.end(), seg, seg + n);
            } else {
                if (carrier < 0) carrier = (int64_t)k;
                put_le(pay, 1, 4);
                put_le(pay, (uint64_t)carrier, 4);
                if (carrier == (int64_t)k)
                    for (int i = 0; i < 128; i++) pay.push_back((uint8_t)(len[2 * i] | (len[2 * i + 1] << 4)));
                for (uint32_t l = 0; l < kLanes; l++) put_le(pay, lane_len[l], 2);
                for (uint32_t l = 0; l < kLanes; l++) {
                    const size_t at = pay.size();
                    pay.resize(at + lane_len[l], 0);
                    uint64_t bit = 0;
                    for (uint32_t j = l; j < n; j += kLanes) {
                        const uint32_t c = code[seg[j]], L = len[seg[j]];
                        for (uint32_t i = L; i-- > 0; bit++)
                            if ((c >> i) & 1u) pay[at + bit / 8] |= (uint8_t)(0x80u >> (bit % 8));
                    }
                }
            }
            pay.resize(aceapex::align16(pay.size()), 0);
        }
    }
    const uint64_t e_len = head + pay.size();
    uint8_t *o = (uint8_t *)calloc(e_len, 1);
    if (!o) return aceapex::kErrNomem;
    set_le(o, 0x45454341u, 4);
    set_le(o + 4, 1, 2);
    set_le(o + 12, kMaxLen, 4);
    set_le(o + 16, raw_len, 8);
    set_le(o + 24, n_seg, 8);
    set_le(o + 32, e_len, 8);
    for (uint64_t i = 0; i < n_seg; i++) {
        set_le(o + 64 + 16 * i, r_off[i], 8);
        set_le(o + 72 + 16 * i, p_off[i], 8);
    }
    if (!pay.empty()) memcpy(o + head, pay.data(), pay.size());
    *out = o;
    *out_len = e_len;
    return aceapex::kOK;
}
