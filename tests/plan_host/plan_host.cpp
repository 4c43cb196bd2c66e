// Host driver for the planner's constant table (paper_2609_29554_gb300/csrc/plan.cpp):
// builds the plan and the DevTable every kernel reads for a few precisions and
// prints them for an exact comparison with the oracle's integers in Python.
//
// Backend code 0 is the p-bit planner, -1 the allocation-free GEMM's planner
// (plan_noalloc, which writes the table directly).
// Output per plan: "plan p K backend S w N WG", then per modulus
// "mod l m y magic invm(hex float) pow16[0..MAXH) Mlow[0..MAXWG)", then
// "Plow Plow[0..MAXWG)".
#include <cstdio>
#include <cstdlib>

#include "ozlu_internal.h"

int main(int argc, char** argv) {
    using namespace ozlu;
    if (argc > 1 && argv[1][0] == 'L') {
        // Eq. (Lhint) seeds: arguments r t M N (quadruples after "L")
        for (int i = 2; i + 3 < argc; i += 4)
            printf("lhint %s %s %s %s %d\n", argv[i], argv[i + 1], argv[i + 2], argv[i + 3],
                   lhint_S(atof(argv[i]), atoi(argv[i + 1]), atoi(argv[i + 2]), atoi(argv[i + 3])));
        return 0;
    }
    for (int i = 1; i + 2 < argc; i += 3) {
        const int p = atoi(argv[i]), K = atoi(argv[i + 1]), be = atoi(argv[i + 2]);
        Plan pl;
        DevTable t;
        int rc;
        if (be == -1) {
            int kpad = 0;
            rc = plan_noalloc(p, K, t, kpad);
        } else if (be == 0) {
            rc = make_plan_mp(p, K, pl);
        } else {
            ozlu_opts o = {};
            o.backend = be;
            rc = make_plan(p, K, &o, pl);
        }
        if (rc) {
            printf("fail %d %d %d %d\n", p, K, be, rc);
            continue;
        }
        if (be != -1) fill_table(pl, t);
        printf("plan %d %d %d %d %d %d %d\n", p, K, be, t.S, t.w, t.N, t.WG);
        for (int l = 0; l < t.N; ++l) {
            printf("mod %d %d %d %u %a", l, t.mod[l], t.y[l], t.magic[l], (double)t.invm[l]);
            for (int j = 0; j < MAXH; ++j) printf(" %u", t.pow16[l][j]);
            for (int w = 0; w < MAXWG; ++w) printf(" %u", t.Mlow[l][w]);
            printf("\n");
        }
        printf("Plow");
        for (int w = 0; w < MAXWG; ++w) printf(" %u", t.Plow[w]);
        printf("\n");
    }
    return 0;
}
