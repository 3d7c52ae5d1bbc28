"""Write the closed-form fixtures (no call into the oracle or the CUDA path)."""
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def grid2d_sigma(N):
    t = [4.0 * math.sin(i * math.pi / (2 * (N + 1))) ** 2 for i in range(1, N + 1)]
    return sorted(math.sqrt(a + b) for a in t for b in t)


if __name__ == "__main__":
    s = grid2d_sigma(32)
    with open(os.path.join(HERE, "grid2d_N32_sigma.txt"), "w") as f:
        f.write("# closed form, 2D grid-difference operator N=32 (2112 x 1024)\n")
        f.write("# smallest 5\n")
        for v in s[:5]:
            f.write(f"{v:.17e}\n")
        f.write("# largest 5\n")
        for v in s[::-1][:5]:
            f.write(f"{v:.17e}\n")
