"""GB300-native batched tensor-network contraction of parameterised circuits."""
