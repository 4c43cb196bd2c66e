// Host driver for the extended-table planner (paper_2609_29554_gb300/csrc/plan.cpp):
// builds the plan and the image of its device tables (build_ext_image) and
// prints sampled entries for an exact comparison with the oracle in Python.
//
// Arguments: triples p K S.  Output per plan: "plan p K S N WG WD w", then for
// every 7th modulus and the last "mod l m y magic c0 c1 c2 pw two32 inv40
// pow32[0] pow32[1] pow32[2] pow32[WD-1] Mw[0] Mw[1] Mw[WG-1]", then
// "P Pw[0] Pw[1] Pw[WG-1]".
#include <cstdio>
#include <cstdlib>

#include "ozlu_internal.h"

int main(int argc, char** argv) {
    using namespace ozlu;
    for (int i = 1; i + 2 < argc; i += 3) {
        const int p = atoi(argv[i]), K = atoi(argv[i + 1]), S = atoi(argv[i + 2]);
        Plan pl;
        if (make_plan_mp_ext(p, K, S, pl)) {
            printf("fail %d %d %d\n", p, K, S);
            continue;
        }
        ExtImage img;
        build_ext_image(pl, img);
        const int N = pl.N, WG = pl.WG, WD = img.WD;
        const uint32_t* w = img.words.data();
        printf("plan %d %d %d %d %d %d %d\n", p, K, S, N, WG, WD, pl.w);
        for (int l = 0; l < N; ++l) {
            if (l % 7 && l != N - 1) continue;
            const unsigned long long inv = (unsigned long long)w[img.o_inv40 + 2 * l] |
                                           ((unsigned long long)w[img.o_inv40 + 2 * l + 1] << 32);
            printf("mod %d %u %u %u %u %u %u %u %u %llu %u %u %u %u %u %u %u\n", l, w[img.o_mod + l],
                   w[img.o_y + l], w[img.o_magic + l], w[img.o_coef + l], w[img.o_coef + N + l],
                   w[img.o_coef + 2 * N + l], w[img.o_pw + l], w[img.o_two32 + l], inv, w[img.o_pow32 + l],
                   w[img.o_pow32 + (size_t)N + l], w[img.o_pow32 + 2 * (size_t)N + l],
                   w[img.o_pow32 + (size_t)(WD - 1) * N + l], w[img.o_Mw + l], w[img.o_Mw + (size_t)N + l],
                   w[img.o_Mw + (size_t)(WG - 1) * N + l]);
        }
        printf("P %u %u %u\n", w[img.o_Pw], w[img.o_Pw + 1], w[img.o_Pw + WG - 1]);
    }
    return 0;
}
