// Drives the batch arena's offset bookkeeping (FreeList in arena.h) from a script on
// standard input, one command per line:
//   reset S      -> "ok"
//   alloc B      -> the offset, or -1 when nothing fits
//   free OFF B   -> "ok"
//   dump         -> "used" then each free block as "offset:length", by offset
#include <cstdio>
#include <cstring>

#include "arena.h"

int main()
{
    ising::FreeList f;
    char cmd[16];
    long long a = 0, b = 0;
    while (std::scanf("%15s", cmd) == 1) {
        if (!std::strcmp(cmd, "reset") && std::scanf("%lld", &a) == 1) {
            f.reset(a);
            std::puts("ok");
        } else if (!std::strcmp(cmd, "alloc") && std::scanf("%lld", &a) == 1) {
            std::printf("%lld\n", (long long)f.alloc(a));
        } else if (!std::strcmp(cmd, "free") && std::scanf("%lld %lld", &a, &b) == 2) {
            f.release(a, b);
            std::puts("ok");
        } else if (!std::strcmp(cmd, "dump")) {
            std::printf("%lld", (long long)f.used);
            for (const auto& kv : f.free_) std::printf(" %lld:%lld", (long long)kv.first, (long long)kv.second);
            std::puts("");
        } else {
            std::printf("bad command %s\n", cmd);
            return 1;
        }
    }
    return 0;
}
