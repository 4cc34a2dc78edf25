"""Host-side check of the search kernel's patch-to-lane-group mapping.

A search block owns a chunk of consecutive patches of one patch row.  Its 8
warps take, pass after pass, groups of G lanes (one patch per group, G = 8
for patch sizes up to 8, 16 above); the groups of a warp take patches `sp`
apart so that their rows fall in different shared-memory banks.  The slot of
warp u (counted over the passes) and group q is (u / sp) sp GPW + u % sp +
sp q, with GPW = 32 / G groups per warp, and a pass is skipped when its
smallest slot is past the chunk's last patch.  This restates that arithmetic
(csrc/bdis_kernels.cu, search_unit) and checks that every slot of every
chunk fill is processed exactly once, for every lane width, stride and pass
count the autotuner can choose.
"""


def spacing(G, S, passes):
    GPW = 32 // G
    sp = (32 // GPW) // S
    sp = 16 if sp >= 16 else 8 if sp >= 8 else 4 if sp >= 4 else 2 if sp >= 2 else 1
    chunk = passes * (256 // G)
    ns = 8 * (chunk // (8 * GPW))
    while ns % sp:
        sp >>= 1
    return sp


def slots_processed(G, S, passes, nk):
    GPW = 32 // G
    sp = spacing(G, S, passes)
    got = []
    for p in range(passes):
        if ((p * 8) // sp) * (sp * GPW) + (p * 8) % sp >= nk:
            break
        for w in range(8):
            uu = p * 8 + w
            for q in range(GPW):
                kk = (uu // sp) * (sp * GPW) + uu % sp + sp * q
                if kk < nk:
                    got.append(kk)
    return got


def test_every_slot_once():
    for G in (8, 16):
        for S in range(1, 17):
            for passes in (1, 2, 3, 4):
                chunk = passes * (256 // G)
                for nk in range(1, chunk + 1):
                    assert sorted(slots_processed(G, S, passes, nk)) == list(range(nk)), \
                        (G, S, passes, nk)


def test_contiguous_skip_would_lose_slots():
    # the skip by a contiguous range [p 8 GPW, (p + 1) 8 GPW) loses slots 8..15
    # when 16 lanes per patch meet stride 1 (groups 16 patches apart)
    G, S, passes, nk = 16, 1, 2, 12
    GPW = 32 // G
    sp = spacing(G, S, passes)
    assert sp == 16
    got = []
    for p in range(passes):
        if p * 8 * GPW >= nk:
            break
        for w in range(8):
            uu = p * 8 + w
            for q in range(GPW):
                kk = (uu // sp) * (sp * GPW) + uu % sp + sp * q
                if kk < nk:
                    got.append(kk)
    assert sorted(got) == list(range(8))
    assert sorted(slots_processed(G, S, passes, nk)) == list(range(nk))
