"""Write edge_counts.json: closed-form edge counts of radius-R pixel graphs.

For a W x H pixel grid, an offset (dx, dy) connects (W - |dx|) * (H - |dy|)
ordered pixel pairs.  Summing over all offsets with 0 < dx^2 + dy^2 <= R^2
gives the directed edge count; half of it is the undirected count.
"""
import json
import os


def counts(W, H, R):
    Ri = int(R)
    offs = [(dx, dy) for dy in range(-Ri, Ri + 1) for dx in range(-Ri, Ri + 1)
            if 0 < dx * dx + dy * dy <= R * R]
    directed = sum((W - abs(dx)) * (H - abs(dy)) for dx, dy in offs)
    n = W * H
    return {"W": W, "H": H, "radius": R, "offsets": len(offs), "n": n,
            "directed": directed, "undirected": directed // 2, "nnz_A": n + directed}


if __name__ == "__main__":
    out = {
        "C1": counts(32, 32, 2.0),
        "C2": counts(481, 321, 3.0),
        "C5": counts(2048, 2048, 2.0),
        "grid128_4nn": counts(128, 128, 1.0),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "edge_counts.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))
