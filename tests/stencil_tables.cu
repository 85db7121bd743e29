// Host program for tests/test_stencil_tables.py: prints the kinetic stencil tables the kernels
// are compiled with (the forward table in the (a, bt) basis, its (P, Q) form and the adjoint
// table), as JSON, so a CPU test can apply them to a state and compare with the oracle's
// operators.  Built with nvcc for the host; no kernel is launched and no GPU is needed.
#include <cstdio>

#include "qlga_adjoint.cuh"
#include "qlga_step2d.cuh"

static void print_table(const char* name, const qlga::KinStencil* tab, bool last) {
    std::printf("\"%s\": [", name);
    for (int v = 0; v < 2; ++v) {
        std::printf("%s[", v ? ", " : "");
        for (int dst = 0; dst < 2; ++dst) {
            std::printf("%s[", dst ? ", " : "");
            for (int src = 0; src < 2; ++src) {
                std::printf("%s[", src ? ", " : "");
                for (int k = 0; k < 9; ++k) std::printf("%s%d", k ? ", " : "", tab[v].g[dst][src][k]);
                std::printf("]");
            }
            std::printf("]");
        }
        std::printf("]");
    }
    std::printf("]%s\n", last ? "" : ",");
}

int main() {
    std::printf("{\n");
    print_table("forward", qlga::kStencil, false);
    print_table("forward_pq", qlga::kStencilPQ, false);
    print_table("adjoint", qlga::kStencilAdj, true);
    std::printf("}\n");
    return 0;
}
