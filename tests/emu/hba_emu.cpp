// hba_emu.cpp -- host emulation of the batch engine, for the test suite only.
//
// Compiles hba_engine.cuh with HBA_EMULATE: every phase of the CTA body runs
// as a loop over thread indices, barriers become no-ops.  The library never
// loads this file's build; the GPU path is the only product path.  The test
// suite uses it to check the engine's logic (chunking, run detection, list
// surgery) against the sequential oracle at sizes and seeds a GPU run could
// not afford, with small CTA widths that force many chunk boundaries.
#define HBA_EMULATE 1
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "hba_engine.cuh"
#include "hba_tlsf.cuh"

using namespace hba;

namespace {
struct Emu {
    Arena ar;
    std::vector<Rec> rec;
    std::vector<uint32_t> scr;
    int nt;
    uint32_t dyn_words = 600;
    int staged = 0;  // write the gathered records straight into the shared-memory layout
    int self = 0;    // the engine gathers its frees' records itself
    int tlsf = 0;    // two-level segregated fit (the engine's POL 1)
    TlsfLists tl;
};

template <int NT, int POL>
void run(Emu* e, const uint64_t* frees, uint32_t nf, uint8_t* st, const uint64_t* sizes,
         uint32_t na, uint64_t* out) {
    Smem<NT, POL>* S = new Smem<NT, POL>();
    if (e->scr.size() < (size_t)SCRATCH_WORDS_PER_FREE * nf) e->scr.resize((size_t)SCRATCH_WORDS_PER_FREE * nf);
    // the gather that a separate grid does on the GPU
    std::vector<uint32_t> gi((size_t)GATHER_WORDS * nf + 1);
    if (!e->self)
        for (uint32_t j = 0; j < nf; ++j)
            gather_free(e->rec.data(), e->ar.arena_bytes, e->ar.G, e->ar.lg, frees[j], gi.data(), nf, j);
    StepArgs a{&e->ar, e->rec.data(), frees, nf, st, sizes, na, out, e->scr.data(), gi.data(), nf, 0, WAIT_NONE, 0,
               e->self ? 1u : 0u, POL ? &e->tl : nullptr};
    // "shared memory": at least what the alloc phase needs, plus a test knob so
    // that both placements of the free-phase arrays run
    const uint32_t words = std::max(alloc_dyn_words<NT, POL>(), e->dyn_words);
    std::vector<uint64_t> dyn(words / 2 + 1);
    uint32_t* d = reinterpret_cast<uint32_t*>(dyn.data());
    if (!e->self && e->staged && nf && stage_fits(nf, words)) {
        // what the gathering CTAs of a cluster do on the GPU
        memcpy(d, gi.data(), sizeof(uint32_t) * GATHER_WORDS * nf);
        a.staged = 1;
    }
    arena_step<NT, POL>(*S, a, d, words);
    delete S;
}
}  // namespace

extern "C" {

void* emu_create(uint64_t arena_bytes, uint64_t min_block, int nt) {
    if (min_block < 8 || (min_block & (min_block - 1))) return nullptr;
    const uint32_t lg = (uint32_t)__builtin_ctzll(min_block);
    const uint64_t a = arena_bytes - arena_bytes % min_block;
    if (a == 0 || (a >> lg) > MAX_GRANULES) return nullptr;
    Emu* e = new Emu();
    e->nt = nt;
    arena_init_host(&e->ar, a, lg, 0);
    e->rec.assign(e->ar.G, Rec{0, 0, 0, 0});
    e->rec[0] = initial_record(e->ar);
    return e;
}

void emu_destroy(void* h) { delete (Emu*)h; }

void emu_set_dyn(void* h, uint32_t words) { ((Emu*)h)->dyn_words = words; }
void emu_set_staged(void* h, int staged) { ((Emu*)h)->staged = staged; }
void emu_set_self(void* h, int self) { ((Emu*)h)->self = self; }

// Two-level segregated fit through the batch engine (POL 1): the lists start
// as one free block, like the TLSF handles'.
void emu_set_tlsf(void* h) {
    Emu* e = (Emu*)h;
    e->tlsf = 1;
    tl_init_host(&e->tl, e->ar.G);
    e->ar.mask = e->tl.flmask;
}

size_t emu_export_tlsf(void* h, uint64_t* buf, size_t cap) {
    Emu* e = (Emu*)h;
    return tl_export(e->ar, e->tl, e->rec.data(), buf, cap);
}

int emu_step(void* h, const uint64_t* frees, uint32_t nf, uint8_t* st, const uint64_t* sizes,
             uint32_t na, uint64_t* out) {
    Emu* e = (Emu*)h;
    if (e->tlsf) {
        switch (e->nt) {
            case 4: run<4, 1>(e, frees, nf, st, sizes, na, out); break;
            case 32: run<32, 1>(e, frees, nf, st, sizes, na, out); break;
            case 256: run<256, 1>(e, frees, nf, st, sizes, na, out); break;
            case 1024: run<1024, 1>(e, frees, nf, st, sizes, na, out); break;
            default: return 1;
        }
        return 0;
    }
    switch (e->nt) {
        case 4: run<4, 0>(e, frees, nf, st, sizes, na, out); break;
        case 32: run<32, 0>(e, frees, nf, st, sizes, na, out); break;
        case 256: run<256, 0>(e, frees, nf, st, sizes, na, out); break;
        case 1024: run<1024, 0>(e, frees, nf, st, sizes, na, out); break;
        default: return 1;
    }
    return 0;
}

// Two-level segregated fit: the per-op functions the GPU warp applies, run
// one request at a time.
struct TlEmu {
    Arena ar;
    TlsfLists L;
    std::vector<Rec> rec;
};

void* emu_tlsf_create(uint64_t arena_bytes, uint64_t min_block) {
    if (min_block < 8 || (min_block & (min_block - 1))) return nullptr;
    const uint32_t lg = (uint32_t)__builtin_ctzll(min_block);
    const uint64_t a = arena_bytes - arena_bytes % min_block;
    if (a == 0 || (a >> lg) > MAX_GRANULES) return nullptr;
    TlEmu* e = new TlEmu();
    arena_init_host(&e->ar, a, lg, 0);
    tl_init_host(&e->L, e->ar.G);
    e->ar.mask = e->L.flmask;
    e->rec.assign(e->ar.G, Rec{0, 0, 0, 0});
    e->rec[0] = initial_record(e->ar);
    return e;
}

void emu_tlsf_destroy(void* h) { delete (TlEmu*)h; }

void emu_tlsf_step(void* h, const uint64_t* frees, uint32_t nf, uint8_t* st, const uint64_t* sizes, uint32_t na,
                   uint64_t* out) {
    TlEmu* e = (TlEmu*)h;
    TlCount c;
    tl_batch_serial(e->L, e->rec.data(), e->ar.arena_bytes, e->ar.G, e->ar.lg, frees, nf, st, sizes, na, out, c);
    tl_apply_counts(e->ar, e->L, c);
}

size_t emu_tlsf_export(void* h, uint64_t* buf, size_t cap) {
    TlEmu* e = (TlEmu*)h;
    return tl_export(e->ar, e->L, e->rec.data(), buf, cap);
}

void emu_tlsf_stats(void* h, uint64_t* out) {
    const Arena& a = ((TlEmu*)h)->ar;
    out[0] = a.alloc_ok;
    out[1] = a.alloc_fail;
    out[2] = a.free_ok;
    out[3] = a.free_fail;
    out[4] = (uint64_t)a.used_g << a.lg;
    out[5] = a.used_blocks;
    out[6] = a.blocks;
    out[7] = a.requested;
    out[8] = a.mask << a.lg;
}

size_t emu_export(void* h, uint64_t* buf, size_t cap) {
    Emu* e = (Emu*)h;
    return export_canonical(e->ar, e->rec.data(), buf, cap);
}

// alloc_ok, alloc_fail, free_ok, free_fail, used_bytes, used_blocks, blocks,
// requested_bytes, bitmask (byte classes)
void emu_stats(void* h, uint64_t* out) {
    Emu* e = (Emu*)h;
    const Arena& a = e->ar;
    out[0] = a.alloc_ok;
    out[1] = a.alloc_fail;
    out[2] = a.free_ok;
    out[3] = a.free_fail;
    out[4] = (uint64_t)a.used_g << a.lg;
    out[5] = a.used_blocks;
    out[6] = a.blocks;
    out[7] = a.requested;
    out[8] = a.mask << a.lg;
}
}
