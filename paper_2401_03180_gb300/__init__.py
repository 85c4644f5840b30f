"""GB300-native ionising-MD hot path (screened pair forces + stochastic
collisional-radiative charge update) behind a small C ABI."""
