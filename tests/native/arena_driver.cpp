// Drives gbr::Arena from a script on stdin and prints the result of every step:
//   "i <size> <bytes>"  -> "A <off>" or "F"      (alloc)
//   "r <off> <bytes>"   -> "R"                    (release)
//   "s"                 -> "S <used> <largest_free> <free_blocks>"
#include <cstdio>
#include <cstring>

#include "arena.h"

int main() {
    gbr::Arena a;
    char op[8];
    unsigned long long x, y;
    while (std::scanf("%7s", op) == 1) {
        if (!std::strcmp(op, "i")) {
            if (std::scanf("%llu", &x) != 1) return 1;
            a.init((size_t)x);
            std::printf("I %zu\n", a.size());
        } else if (!std::strcmp(op, "a")) {
            if (std::scanf("%llu", &x) != 1) return 1;
            size_t off = 0;
            if (a.alloc((size_t)x, &off)) std::printf("A %zu\n", off);
            else std::printf("F\n");
        } else if (!std::strcmp(op, "r")) {
            if (std::scanf("%llu %llu", &x, &y) != 2) return 1;
            a.release((size_t)x, (size_t)y);
            std::printf("R\n");
        } else if (!std::strcmp(op, "s")) {
            std::printf("S %zu %zu %zu\n", a.used(), a.largest_free(), a.free_blocks());
        }
    }
    return 0;
}
