// emu.cu -- TEST HARNESS: the library's routing functions compiled for the
// host, so the CPU suite can check their logic against the oracle without a
// GPU.  Not part of the library and never loaded by it; the GPU tests remain
// the parity tests proper.
#include <algorithm>
#include <cstdint>
#include <utility>
#include <vector>

#include "ss_cw.cuh"
#include "ss_pack.cuh"
#include "ss_rw.cuh"
#include "ss_rwc.cuh"
#include "ss_sliced.cuh"
#include "ss_submaze.cuh"
#include "ss_unequal.cuh"
#include "ss_verify.cuh"

using namespace ssk;

namespace {

// staged: the pair's words read as the pipelined kernel reads them from
// its stage (SmemSeqPad: whatever follows the pair is read as is).
template <int E>
int exact_one(const uint32_t *q, const uint32_t *r, int m, bool staged)
{
    const int w16 = (m + 15) / 16;
    if (staged)
        return rw_route<E, true>(SmemSeqPad{q}, SmemSeqPad{r}, m, E,
                                 0xffffffffu);
    return rw_route<E, true>(GlobalSeq{q, w16}, GlobalSeq{r, w16}, m, E,
                             0xffffffffu);
}

template <int... Es>
int exact_dispatch(int E, const uint32_t *q, const uint32_t *r, int m,
                   bool staged, std::integer_sequence<int, Es...>)
{
    int out = -100;
    ((E == Es ? (out = exact_one<Es>(q, r, m, staged), 0) : 0), ...);
    return out;
}

template <int E>
int cols_one(const uint32_t *q, const uint32_t *r, int m, bool staged)
{
    const int w16 = (m + 15) / 16;
    if constexpr (E >= 1 && E <= 31) {
        if (staged)
            return rw_route_cols<E>(SmemSeqPad{q}, SmemSeqPad{r}, m,
                                    0xffffffffu);
        return rw_route_cols<E>(GlobalSeq{q, w16}, GlobalSeq{r, w16}, m,
                                0xffffffffu);
    } else {
        return -100;
    }
}

template <int... Es>
int cols_dispatch(int E, const uint32_t *q, const uint32_t *r, int m,
                  bool staged, std::integer_sequence<int, Es...>)
{
    int out = -100;
    ((E == Es ? (out = cols_one<Es>(q, r, m, staged), 0) : 0), ...);
    return out;
}

template <int E>
int uq_exact_one(const uint32_t *q, int mQ, const uint32_t *r, int mR)
{
    const GlobalSeq Q{q, (mQ + 15) / 16}, R{r, (mR + 15) / 16};
    return unequal_route_exact<E>(Q, mQ, R, mR, 0xffffffffu);
}

template <int... Es>
int uq_exact_dispatch(int E, const uint32_t *q, int mQ, const uint32_t *r,
                      int mR, std::integer_sequence<int, Es...>)
{
    int out = -100;
    ((E == Es ? (out = uq_exact_one<Es>(q, mQ, r, mR), 0) : 0), ...);
    return out;
}

template <int EMAX>
int runtime_one(const uint32_t *q, const uint32_t *r, int m, int E)
{
    const int w16 = (m + 15) / 16;
    return rw_route<EMAX, false>(GlobalSeq{q, w16}, GlobalSeq{r, w16}, m, E,
                                 0xffffffffu);
}

template <int K>
int cw_one(const uint32_t *q, const uint32_t *r, int m, int E)
{
    const int Ee = eff_threshold(m, E);
    const CwLayout L = CwLayout::of(m, Ee);
    std::vector<uint32_t> sm(L.words());
    cw_stage(sm.data(), L, q, r, m, 0, 1);
    const int nwords = (2 * Ee + 1 + 31) >> 5;
    int c = 0, count = 0;
    for (;;) {
        int pstar = -1;
        for (int w = 0; w < nwords; ++w)
            pstar = imax(pstar, cw_word<K>(sm.data(), L, m, Ee, c, w));
        if (pstar >= m)
            break;
        ++count;
        if (count > E)
            break;
        c = pstar + 1;
    }
    return count;
}

template <int... Es>
int ed_dispatch(int E, const uint32_t *q, const uint32_t *r, int m,
                std::integer_sequence<int, Es...>)
{
    int out = -100;
    const int w16 = (m + 15) / 16;
    ((E == Es ? (out = ed_banded<Es>(q, r, m, w16), 0) : 0), ...);
    return out;
}

// Sub-maze approximate mode: t-column sub-mazes, at most y obstacles each.
// form 0: the kernels' choice per class; 1: the row-wise routine at every
// class; 2: the column walk at every class it supports (-2 above).
template <class Seq>
int submaze_form(const Seq &Q, const Seq &R, int m, int E, int t, int y,
                 int form)
{
    const int Ee = eff_threshold(m, E);
    if (form == 0) {
        if (Ee <= 3)
            return submaze_route<3>(Q, R, m, E, t, y, 0xffffffffu);
        if (Ee <= 7)
            return submaze_route_cols<7>(Q, R, m, E, t, y);
        if (Ee <= 15)
            return submaze_route_cols<15>(Q, R, m, E, t, y);
        return submaze_route<31>(Q, R, m, E, t, y, 0xffffffffu);
    }
    if (form == 1) {
        if (Ee <= 3)
            return submaze_route<3>(Q, R, m, E, t, y, 0xffffffffu);
        if (Ee <= 7)
            return submaze_route<7>(Q, R, m, E, t, y, 0xffffffffu);
        if (Ee <= 15)
            return submaze_route<15>(Q, R, m, E, t, y, 0xffffffffu);
        return submaze_route<31>(Q, R, m, E, t, y, 0xffffffffu);
    }
    if (Ee <= 1)
        return submaze_route_cols<1>(Q, R, m, E, t, y);
    if (Ee <= 3)
        return submaze_route_cols<3>(Q, R, m, E, t, y);
    if (Ee <= 7)
        return submaze_route_cols<7>(Q, R, m, E, t, y);
    if (Ee <= 15)
        return submaze_route_cols<15>(Q, R, m, E, t, y);
    return -2;
}

// One group of the bit-sliced layout in host memory (the kernel's loads).
struct HostSliced {
    const uint32_t *q, *r;
    int64_t G, g;
    void load(const uint32_t *base, int blk, uint32_t (&lo)[4],
              uint32_t (&hi)[4]) const
    {
        const uint32_t *p = base + ((int64_t)blk * G + g) * 8;
        for (int x = 0; x < 4; ++x) {
            lo[x] = p[x];
            hi[x] = p[4 + x];
        }
    }
    void query(int blk, int nb, uint32_t (&lo)[4], uint32_t (&hi)[4]) const
    {
        if (blk < 0 || blk >= nb) {
            for (int x = 0; x < 4; ++x)
                lo[x] = hi[x] = 0u;
            return;
        }
        load(q, blk, lo, hi);
    }
    void ref(int blk, uint32_t (&lo)[4], uint32_t (&hi)[4]) const
    {
        load(r, blk, lo, hi);
    }
    void prefetch(int, int, int, int) const {}
};

template <int E>
void sliced_groups(const uint32_t *q, const uint32_t *r, int64_t n, int m,
                   uint8_t *acc, int32_t *obs)
{
    const int64_t G = (n + 31) / 32;
    for (int64_t g = 0; g < G; ++g) {
        const int np = (int)std::min<int64_t>(32, n - 32 * g);
        const uint32_t pad = np >= 32 ? 0u : 0xffffffffu << np;
        using Ed = SlicedEdges<E>;
        constexpr int WW = SlicedShape<E>::WW;
        const Ed ed(m);
        std::vector<uint32_t> vtab(Ed::kRows * WW);
        for (int i = 0; i < ed.rows() * WW; ++i)
            vtab[i] = Ed::valid(ed.block_of(i / WW), i % WW, m);
        SlicedCount<E> cnt;
        sliced_walk<E>(HostSliced{q, r, G, g}, m, pad, cnt, vtab.data(), 1u);
        uint32_t cb[SlicedShape<E>::NB];
        cnt.bits(cb);
        for (int i = 0; i < np; ++i) {
            obs[32 * g + i] = sliced_count<E>(cb, i);
            acc[32 * g + i] = (uint8_t)(((~cnt.done()) >> i) & 1u);
        }
    }
}

// Reads of mQ bases against references of mR (mQ != mR) over the sliced
// layout, every group, with the free-end rule.
template <int E>
void sliced_free_groups(const uint32_t *q, const uint32_t *r, int64_t n,
                        int mQ, int mR, uint8_t *acc, int32_t *obs)
{
    const int64_t G = (n + 31) / 32;
    using Ed = SlicedEdges<E>;
    constexpr int WW = SlicedShape<E>::WW;
    const Ed ed(mQ, mR);
    std::vector<uint32_t> vtab(Ed::kRowsFree * WW);
    for (int i = 0; i < ed.rows() * WW; ++i)
        vtab[i] = Ed::entry(ed.block_of(i / WW), i % WW, mQ, mQ != mR);
    for (int64_t g = 0; g < G; ++g) {
        const int np = (int)std::min<int64_t>(32, n - 32 * g);
        const uint32_t pad = np >= 32 ? 0u : 0xffffffffu << np;
        SlicedCount<E> cnt;
        sliced_walk2<E, true>(HostSliced{q, r, G, g}, mQ, mR, pad, cnt,
                              vtab.data(), 1u);
        uint32_t cb[SlicedShape<E>::NB];
        cnt.bits(cb);
        for (int i = 0; i < np; ++i) {
            obs[32 * g + i] = sliced_count<E>(cb, i);
            acc[32 * g + i] = (uint8_t)(((~cnt.done()) >> i) & 1u);
        }
    }
}

template <int... Es>
int sliced_free_dispatch(int E, const uint32_t *q, const uint32_t *r,
                         int64_t n, int mQ, int mR, uint8_t *acc,
                         int32_t *obs, std::integer_sequence<int, Es...>)
{
    int out = -100;
    ((E == Es ? (sliced_free_groups<Es>(q, r, n, mQ, mR, acc, obs), out = 0)
              : 0),
     ...);
    return out;
}

template <int E>
void sliced_sub_groups(const uint32_t *q, const uint32_t *r, int64_t n, int m,
                       int t, int y, uint8_t *acc, int32_t *obs)
{
    const int64_t G = (n + 31) / 32;
    using Ed = SlicedEdges<E>;
    constexpr int WW = SlicedShape<E>::WW;
    const Ed ed(m);
    std::vector<uint32_t> vtab(Ed::kRows * WW);
    for (int i = 0; i < ed.rows() * WW; ++i)
        vtab[i] = Ed::valid(ed.block_of(i / WW), i % WW, m);
    for (int64_t g = 0; g < G; ++g) {
        const int np = (int)std::min<int64_t>(32, n - 32 * g);
        const uint32_t pad = np >= 32 ? 0u : 0xffffffffu << np;
        SlicedCount<E> cnt;
        sliced_walk<E>(HostSliced{q, r, G, g}, m, pad, cnt, vtab.data(), 1u,
                       SlicedSubMaze<E>(t, y));
        uint32_t cb[SlicedShape<E>::NB];
        cnt.bits(cb);
        for (int i = 0; i < np; ++i) {
            obs[32 * g + i] = sliced_count<E>(cb, i);
            acc[32 * g + i] = (uint8_t)(((~cnt.done()) >> i) & 1u);
        }
    }
}

template <int... Es>
int sliced_sub_dispatch(int E, const uint32_t *q, const uint32_t *r,
                        int64_t n, int m, int t, int y, uint8_t *acc,
                        int32_t *obs, std::integer_sequence<int, Es...>)
{
    int out = -100;
    ((E == Es ? (sliced_sub_groups<Es>(q, r, n, m, t, y, acc, obs), out = 0)
              : 0),
     ...);
    return out;
}

template <int... Es>
int sliced_dispatch(int E, const uint32_t *q, const uint32_t *r, int64_t n,
                    int m, uint8_t *acc, int32_t *obs,
                    std::integer_sequence<int, Es...>)
{
    int out = -100;
    ((E == Es ? (sliced_groups<Es>(q, r, n, m, acc, obs), out = 0) : 0), ...);
    return out;
}

template <int I>
void store_set_host(const SlicedTracks<> &, int64_t, int, uint8_t **,
                    int32_t **)
{
}

template <int I, int E, int... R>
void store_set_host(const SlicedTracks<E, R...> &t, int64_t p0, int np,
                    uint8_t **acc, int32_t **obs)
{
    uint32_t cb[SlicedShape<E>::NB];
    t.head.cnt.bits(cb);
    for (int i = 0; i < np; ++i) {
        obs[I][p0 + i] = sliced_count<E>(cb, i);
        acc[I][p0 + i] = (uint8_t)(((~t.head.cnt.done()) >> i) & 1u);
    }
    store_set_host<I + 1>(t.tail, p0, np, acc, obs);
}

template <int EMAX, int... Es>
void sliced_set_groups(const uint32_t *q, const uint32_t *r, int64_t n, int m,
                       uint8_t **acc, int32_t **obs)
{
    const int64_t G = (n + 31) / 32;
    using Ed = SlicedEdges<EMAX>;
    constexpr int WW = SlicedShape<EMAX>::WW;
    const Ed ed(m);
    std::vector<uint32_t> vtab(Ed::kRows * WW);
    for (int i = 0; i < ed.rows() * WW; ++i)
        vtab[i] = Ed::valid(ed.block_of(i / WW), i % WW, m);
    for (int64_t g = 0; g < G; ++g) {
        const int np = (int)std::min<int64_t>(32, n - 32 * g);
        const uint32_t pad = np >= 32 ? 0u : 0xffffffffu << np;
        SlicedTracks<Es...> t;
        sliced_walk_set<EMAX>(HostSliced{q, r, G, g}, m, pad, t, vtab.data(),
                              1u);
        store_set_host<0>(t, 32 * g, np, acc, obs);
    }
}

}  // namespace

extern "C" {

// Several thresholds in one pass over the sliced layout (the sweep's shared
// pass) for the sets {0,2,4}, {0,1,2,3,4}, {1,3}, {3,4} (which = 0..3):
// acc[i], obs[i] get the set's i-th threshold.
int emu_sliced_set(const uint32_t *q, const uint32_t *r, int64_t n, int m,
                   int which, uint8_t **acc, int32_t **obs)
{
    switch (which) {
    case 0: sliced_set_groups<4, 0, 2, 4>(q, r, n, m, acc, obs); return 0;
    case 1: sliced_set_groups<4, 0, 1, 2, 3, 4>(q, r, n, m, acc, obs); return 0;
    case 2: sliced_set_groups<3, 1, 3>(q, r, n, m, acc, obs); return 0;
    case 3: sliced_set_groups<4, 3, 4>(q, r, n, m, acc, obs); return 0;
    default: return -100;
    }
}

// The bit-sliced walk over every group of a sliced layout (n pairs of
// length m): the plain sliced launch's results.  Returns -100 if E is not
// built.
int emu_sliced(const uint32_t *q, const uint32_t *r, int64_t n, int m, int E,
               uint8_t *acc, int32_t *obs)
{
    return sliced_dispatch(E, q, r, n, m, acc, obs,
                           std::make_integer_sequence<int, 32>{});
}

// Reads of mQ bases against references of mR bases (mQ != mR) over the
// sliced layout, with the free-end rule, every group.  Returns -100 if E is
// not built, -1 for equal lengths.
int emu_sliced_free(const uint32_t *q, const uint32_t *r, int64_t n, int mQ,
                    int mR, int E, uint8_t *acc, int32_t *obs)
{
    if (mQ == mR)
        return -1;
    return sliced_free_dispatch(E, q, r, n, mQ, mR, acc, obs,
                                std::make_integer_sequence<int, 32>{});
}

// The sub-maze mode over the sliced layout (sub-mazes of t columns, at most
// y segments each), every group.  Returns -100 if E is not built.
int emu_sliced_submaze(const uint32_t *q, const uint32_t *r, int64_t n, int m,
                       int E, int t, int y, uint8_t *acc, int32_t *obs)
{
    return sliced_sub_dispatch(E, q, r, n, m, t, y, acc, obs,
                               std::make_integer_sequence<int, 16>{});
}

// The warp transpose of the sliced packer, the 32 lanes simulated in turn:
// v[32] in, out[32] out (lane r gets bit r of every lane's word).
void emu_transpose32(const uint32_t *v, uint32_t *out)
{
    uint32_t a[32];
    for (int i = 0; i < 32; ++i)
        a[i] = v[i];
    for (int d = 16; d >= 1; d >>= 1) {
        uint32_t b[32];
        for (int lane = 0; lane < 32; ++lane)
            b[lane] = transpose_level(a[lane], a[lane ^ d], lane, d);
        for (int i = 0; i < 32; ++i)
            a[i] = b[i];
    }
    for (int i = 0; i < 32; ++i)
        out[i] = a[i];
}

// Pack arithmetic: 16 ASCII bytes -> packed word, error bits.
uint32_t emu_pack_chunk(const uint8_t *b16, uint32_t *err)
{
    uint32_t x[4];
    for (int q = 0; q < 4; ++q)
        x[q] = (uint32_t)b16[4 * q] | ((uint32_t)b16[4 * q + 1] << 8) |
               ((uint32_t)b16[4 * q + 2] << 16) |
               ((uint32_t)b16[4 * q + 3] << 24);
    uint32_t e = 0;
    const uint32_t r = pack_chunk(x, e);
    *err = e;
    return r;
}

// The sliced packer's arithmetic: 16 ASCII bytes -> 32 code bits in base
// order (base t at bits 2t, 2t+1), error bits.
uint32_t emu_pack_chunk_pairs(const uint8_t *b16, uint32_t *err)
{
    uint32_t x[4];
    for (int q = 0; q < 4; ++q)
        x[q] = (uint32_t)b16[4 * q] | ((uint32_t)b16[4 * q + 1] << 8) |
               ((uint32_t)b16[4 * q + 2] << 16) |
               ((uint32_t)b16[4 * q + 3] << 24);
    uint32_t e = 0;
    const uint32_t r = pack_chunk_pairs(x, e);
    *err = e;
    return r;
}

uint32_t emu_pack_window(uint32_t c0, uint32_t c1, uint32_t r)
{
    return pack_window(c0, c1, r);
}

// Pairs of different lengths: count, or -2 when more than 31 rows.
int emu_unequal(const uint32_t *q, int mQ, const uint32_t *r, int mR, int E)
{
    const GlobalSeq Q{q, (mQ + 15) / 16}, R{r, (mR + 15) / 16};
    const int rows = unequal_rows(mQ, mR, E);
    if (rows < 0)
        return 0;
    if (rows <= 3)
        return rw_route2<3>(Q, mQ, R, mR, E, 0xffffffffu);
    if (rows <= 7)
        return rw_route2_cols<7>(Q, mQ, R, mR, E);
    if (rows <= 15)
        return rw_route2_cols<15>(Q, mQ, R, mR, E);
    if (rows <= 31)
        return rw_route2<31>(Q, mQ, R, mR, E, 0xffffffffu);
    return -2;
}

// The unequal-length routine of the kernel's class for the pair's rows,
// reading the pair in place from buffers whose words continue past the
// sequences (as in a shared-memory slot): count, or -2 past 31 rows.
int emu_unequal_staged(const uint32_t *q, int mQ, const uint32_t *r, int mR,
                       int E)
{
    const SmemSeqPad Q{q}, R{r};
    const int rows = unequal_rows(mQ, mR, E);
    if (rows < 0)
        return 0;
    if (rows <= 3)
        return unequal_route<3>(Q, mQ, R, mR, E, 0xffffffffu);
    if (rows <= 7)
        return unequal_route<7>(Q, mQ, R, mR, E, 0xffffffffu);
    if (rows <= 15)
        return unequal_route<15>(Q, mQ, R, mR, E, 0xffffffffu);
    if (rows <= 31)
        return unequal_route<31>(Q, mQ, R, mR, E, 0xffffffffu);
    return -2;
}

// The exact-threshold routine of the uniform-threshold launch.
int emu_unequal_exact(const uint32_t *q, int mQ, const uint32_t *r, int mR,
                      int E)
{
    if (unequal_rows(mQ, mR, E) < 0)
        return 0;
    return uq_exact_dispatch(E, q, mQ, r, mR,
                             std::make_integer_sequence<int, 32>{});
}

// Both unequal-length routines at every class they support (form 0:
// row-wise, 1: column walk; -2 past the class table or the form's rows).
int emu_unequal_form(const uint32_t *q, int mQ, const uint32_t *r, int mR,
                     int E, int form)
{
    const GlobalSeq Q{q, (mQ + 15) / 16}, R{r, (mR + 15) / 16};
    const int rows = unequal_rows(mQ, mR, E);
    if (rows < 0)
        return 0;
    if (form == 1) {
        if (rows <= 1)
            return rw_route2_cols<1>(Q, mQ, R, mR, E);
        if (rows <= 3)
            return rw_route2_cols<3>(Q, mQ, R, mR, E);
        if (rows <= 7)
            return rw_route2_cols<7>(Q, mQ, R, mR, E);
        if (rows <= 15)
            return rw_route2_cols<15>(Q, mQ, R, mR, E);
        return -2;
    }
    if (rows <= 3)
        return rw_route2<3>(Q, mQ, R, mR, E, 0xffffffffu);
    if (rows <= 7)
        return rw_route2<7>(Q, mQ, R, mR, E, 0xffffffffu);
    if (rows <= 15)
        return rw_route2<15>(Q, mQ, R, mR, E, 0xffffffffu);
    if (rows <= 31)
        return rw_route2<31>(Q, mQ, R, mR, E, 0xffffffffu);
    return -2;
}

int emu_submaze(const uint32_t *q, const uint32_t *r, int m, int E, int t,
                int y)
{
    const int w16 = (m + 15) / 16;
    return submaze_form(GlobalSeq{q, w16}, GlobalSeq{r, w16}, m, E, t, y, 0);
}

int emu_submaze_rows(const uint32_t *q, const uint32_t *r, int m, int E, int t,
                     int y)
{
    const int w16 = (m + 15) / 16;
    return submaze_form(GlobalSeq{q, w16}, GlobalSeq{r, w16}, m, E, t, y, 1);
}

int emu_submaze_cols(const uint32_t *q, const uint32_t *r, int m, int E, int t,
                     int y)
{
    const int w16 = (m + 15) / 16;
    return submaze_form(GlobalSeq{q, w16}, GlobalSeq{r, w16}, m, E, t, y, 2);
}

// The same over staged words as the pipelined kernels read them: whatever
// follows the pair's words (another pair, the R plane) is read as is.
int emu_submaze_staged(const uint32_t *q, const uint32_t *r, int m, int E,
                       int t, int y, int form)
{
    return submaze_form(SmemSeqPad{q}, SmemSeqPad{r}, m, E, t, y, form);
}

// Banded edit distance of the accuracy harness: min(ED, E+1), E <= 31.
int emu_ed(const uint32_t *q, const uint32_t *r, int m, int E)
{
    return ed_dispatch(E, q, r, m, std::make_integer_sequence<int, 32>{});
}

// Plain-kernel routine with compile-time E (0..31).
int emu_rw_exact(const uint32_t *q, const uint32_t *r, int m, int E)
{
    return exact_dispatch(E, q, r, m, false,
                          std::make_integer_sequence<int, 32>{});
}

// Column-at-a-time routine (E = 1..15).
int emu_rw_cols(const uint32_t *q, const uint32_t *r, int m, int E)
{
    return cols_dispatch(E, q, r, m, false,
                         std::make_integer_sequence<int, 32>{});
}

// Both, over staged words (cols: the column walk, else row-wise).
int emu_rw_staged(const uint32_t *q, const uint32_t *r, int m, int E,
                  int cols)
{
    if (cols)
        return cols_dispatch(E, q, r, m, true,
                             std::make_integer_sequence<int, 32>{});
    return exact_dispatch(E, q, r, m, true,
                          std::make_integer_sequence<int, 32>{});
}

// Bucketed row-wise routine: runtime E <= EMAX (1, 3, 7, 15, 31).
int emu_rw_runtime(const uint32_t *q, const uint32_t *r, int m, int E,
                   int emax)
{
    switch (emax) {
    case 1: return runtime_one<1>(q, r, m, E);
    case 3: return runtime_one<3>(q, r, m, E);
    case 7: return runtime_one<7>(q, r, m, E);
    case 15: return runtime_one<15>(q, r, m, E);
    case 31: return runtime_one<31>(q, r, m, E);
    default: return -100;
    }
}

// Column-wise routine with subgrid width K (4, 8, 16), serial group max.
int emu_cw(const uint32_t *q, const uint32_t *r, int m, int E, int K)
{
    switch (K) {
    case 4: return cw_one<4>(q, r, m, E);
    case 8: return cw_one<8>(q, r, m, E);
    case 16: return cw_one<16>(q, r, m, E);
    default: return -100;
    }
}

// Class of a pair under the default tuning (for coverage checks).
int emu_class_of(int m, int E) { return class_of(m, E); }

}  // extern "C"
