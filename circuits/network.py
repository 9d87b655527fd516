"""Circuit -> tensor network (Section 2.2.1).

Each qudit wire carries an integer label that is renewed every time a gate
acts on it.  Tensors are row-major with labels[0] the slowest index:
  * initial state of qudit q:   rank 1, labels [w]            (|0> or a squeezed vector)
  * 1-qudit gate U on q:        rank 2, labels [new, old]     = U[out, in]
  * 2-qudit gate U on (q1, q2): rank 4, labels [n1, n2, o1, o2] = U reshaped (d,d,d,d)
The final label of every wire is an open leg; an amplitude <x| fixes open leg
q to the digit x_q (the bra of Section 2.2.1).
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np

from .rqc import Circuit


@dataclass
class TensorNetwork:
    labels: List[List[int]] = field(default_factory=list)
    data: List[np.ndarray] = field(default_factory=list)     # complex128, shape = dims
    open_labels: List[int] = field(default_factory=list)     # one per qudit, qudit order
    dim: int = 2
    gate_tensor: List[int] = field(default_factory=list)     # circuit gate index -> tensor id

    @property
    def n_tensors(self) -> int:
        return len(self.data)

    def dims(self, t: int) -> List[int]:
        return list(self.data[t].shape)

    def as_complex64(self) -> "TensorNetwork":
        """The same network with every tensor rounded to complex64 (the values the
        CUDA path receives); the oracle takes these upcast to complex128."""
        return TensorNetwork([list(l) for l in self.labels],
                             [np.asarray(x, dtype=np.complex64).astype(np.complex128)
                              for x in self.data],
                             list(self.open_labels), self.dim, list(self.gate_tensor))


def circuit_to_network(circ: Circuit) -> TensorNetwork:
    d = circ.d
    tn = TensorNetwork(dim=d)
    next_label = 0
    wire = []
    for q in range(circ.n):
        wire.append(next_label)
        tn.labels.append([next_label])
        tn.data.append(np.array(circ.initial[q], dtype=np.complex128).reshape(d))
        next_label += 1
    for g in circ.gates:
        k = len(g.qubits)
        new = list(range(next_label, next_label + k))
        next_label += k
        old = [wire[q] for q in g.qubits]
        tn.gate_tensor.append(len(tn.data))
        tn.labels.append(new + old)
        tn.data.append(np.array(g.matrix, dtype=np.complex128).reshape((d,) * (2 * k)))
        for q, lab in zip(g.qubits, new):
            wire[q] = lab
    tn.open_labels = list(wire)
    return tn
